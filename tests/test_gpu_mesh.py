"""Marching cubes (Sec. 4.6) through the C-ABI against the oracle.

Both sides read the same FP32 indicator (seeded or analytic fields set through
tgv_set_field, frozen values given at creation) and take every decision in FP32
with the same operation order, so the meshes must be identical: vertex
positions bit for bit, triangles index for index.  A solved field is compared
with the oracle's own solve by properties (counts, closedness, geometry).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2107_14790_b300 import tgv
from tests.test_oracle_mesh import centres, closed_oriented

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2107_14790_b300 import build
    build.build()
    assert torch.cuda.is_available()
    tgv.lib()


def gpu_mesh(desc, u_active):
    with tgv.Domain([desc], nbins=8, stream=torch.cuda.current_stream().cuda_stream) as dom:
        dom.set_field(0, "u", u_active.reshape(-1, 1).astype(np.float32))
        return dom.mesh(0)


def same_mesh(desc, u_all):
    nb = desc.nbricks
    V, T = gpu_mesh(desc, u_all[:512 * nb])
    Vo, To = oracle.mesh(desc, u_all)
    np.testing.assert_array_equal(V, Vo)
    np.testing.assert_array_equal(T, To)
    return V, T


def test_sphere_field_identical():
    d = synth.DomainDesc(np.zeros(3), 1.0 / 40, synth.dense_bricks(5))
    X, _ = centres(d)
    u = (np.linalg.norm(X - 0.5, axis=1) - 0.3).astype(np.float32)
    V, T = same_mesh(d, u)
    assert len(T) > 5000 and closed_oriented(T)


@pytest.mark.parametrize("seed,amp", [(0, 1.2), (5, 5.0), (9, 2.5)])
def test_noisy_fields_identical(seed, amp):
    """Many four-crossing faces and centroid fans."""
    rng = np.random.default_rng(seed)
    d = synth.DomainDesc(np.zeros(3), 1.0 / 32, synth.dense_bricks(4))
    X, _ = centres(d)
    u = (np.linalg.norm(X - 0.5, axis=1) - 0.3 + rng.uniform(-1, 1, len(X)) * amp / 32).astype(np.float32)
    V, T = same_mesh(d, u)
    assert closed_oriented(T)


def test_ragged_domain_with_frozen_bricks_identical():
    """Holes, negative brick coordinates and frozen bricks whose u supplies corners."""
    rng = np.random.default_rng(11)
    box = synth.dense_bricks(6, 5, 4, offset=(-3, -2, 1))
    keep = rng.random(len(box)) > 0.2
    act, rest = box[keep], box[~keep]
    frz = rest[: len(rest) // 2]
    d0 = synth.DomainDesc(np.array([0.1, -0.2, 0.05]), 1.0 / 50, act, frozen=frz)
    Xa, _ = centres(d0)
    Xf, _ = centres(d0, frozen=True)
    def field(X):
        return (np.sin(9 * X[:, 0]) * np.cos(7 * X[:, 1]) + 0.6 * np.sin(11 * X[:, 2] + 1.0) - 0.1).astype(np.float32)
    fu = field(Xf).reshape(-1, 512)
    d = synth.DomainDesc(d0.origin, d0.h, act, frozen=frz, frozen_u=fu)
    u_all = np.concatenate([field(Xa), fu.reshape(-1)])
    V, T = same_mesh(d, u_all)
    assert len(T) > 5000


def test_repeated_extraction_on_one_domain():
    """The same domain meshed again after its field changes (more, then fewer crossing
    cells, then none) gives each field's own mesh: the scratch sized by the previous
    extraction is reused or regrown, never read stale."""
    d = synth.DomainDesc(np.zeros(3), 1.0 / 32, synth.dense_bricks(4))
    X, _ = centres(d)
    rng = np.random.default_rng(3)
    sphere = (np.linalg.norm(X - 0.5, axis=1) - 0.3).astype(np.float32)
    noisy = (sphere + rng.uniform(-1, 1, len(X)) * 4.0 / 32).astype(np.float32)
    small = (np.linalg.norm(X - 0.5, axis=1) - 0.1).astype(np.float32)
    with tgv.Domain([d], nbins=8, stream=torch.cuda.current_stream().cuda_stream) as dom:
        for u in (sphere, noisy, small, np.ones_like(sphere), sphere):
            dom.set_field(0, "u", u.reshape(-1, 1))
            V, T = dom.mesh(0)
            Vo, To = oracle.mesh(d, u)
            np.testing.assert_array_equal(V, Vo)
            np.testing.assert_array_equal(T, To)


def test_chunks_with_frozen_halos_mesh_without_seams():
    """A domain cut into two chunks along x, each seeing the other's border bricks as
    frozen bricks with their u: the two meshes together are the whole domain's mesh,
    triangle for triangle with bit-identical coordinates, and no triangle is made twice
    (a cell belongs to the chunk of its lower corner)."""
    rng = np.random.default_rng(21)
    full = synth.DomainDesc(np.zeros(3), 1.0 / 32, synth.dense_bricks(4))
    def field(X):
        return (np.linalg.norm(X - 0.5, axis=1) - 0.3 + rng.uniform(-1, 1, len(X)) * 1.5 / 32).astype(np.float32)
    X, g = centres(full)
    u_full = field(X)
    lookup = {tuple(v): u_full[i] for i, v in enumerate(g.tolist())}
    def chunk(active, frozen):
        d0 = synth.DomainDesc(full.origin, full.h, active, frozen=frozen)
        _, gf = centres(d0, frozen=True)
        fu = np.array([lookup[tuple(v)] for v in gf.tolist()], np.float32).reshape(-1, 512)
        d = synth.DomainDesc(full.origin, full.h, active, frozen=frozen, frozen_u=fu)
        _, ga = centres(d)
        ua = np.array([lookup[tuple(v)] for v in ga.tolist()], np.float32)
        return gpu_mesh(d, ua)
    def triangles(V, T):
        return {V[t].tobytes() for t in T}
    b = full.bricks
    lo, hi = b[b[:, 0] < 2], b[b[:, 0] >= 2]
    tri_a = triangles(*chunk(lo, b[b[:, 0] == 2]))
    tri_b = triangles(*chunk(hi, np.zeros((0, 3), np.int32)))
    V, T = gpu_mesh(full, u_full)
    whole = triangles(V, T)
    assert len(whole) == len(T) and len(T) > 1000
    assert not (tri_a & tri_b)
    assert tri_a | tri_b == whole


def test_empty_and_state_errors():
    d = synth.DomainDesc(np.zeros(3), 1.0 / 16, synth.dense_bricks(2))
    with tgv.Domain([d], nbins=8, stream=torch.cuda.current_stream().cuda_stream) as dom:
        assert tgv.lib().tgv_copy_mesh(dom.handle, None, 0, None, 0) == 6  # STATE: nothing extracted yet
        dom.set_field(0, "u", np.ones((d.nvox, 1), np.float32))
        V, T = dom.mesh(0)
        assert V.shape == (0, 3) and T.shape == (0, 3)
    # a level without active bricks extracts an empty mesh too
    d2 = synth.DomainDesc(np.zeros(3), 1.0 / 16, np.zeros((0, 3), np.int32))
    with tgv.Domain([d, d2], nbins=8, stream=torch.cuda.current_stream().cuda_stream) as dom:
        V, T = dom.mesh(1)
        assert V.shape == (0, 3) and T.shape == (0, 3)


def test_solved_sphere_mesh(sphere_scene):
    """After 200 iterations on the sphere scene: a closed mesh near radius 0.35 whose
    counts agree with the mesh of the oracle's FP64 solve (rounded to FP32)."""
    sc = sphere_scene
    with tgv.Domain([sc.domain], nbins=sc.nbins, stream=torch.cuda.current_stream().cuda_stream) as dom:
        dom.accumulate(0, sc.cameras, torch.from_numpy(np.stack(sc.depths)).cuda())
        dom.solve(0, sc.iterations)
        V, T = dom.mesh(0)
    orc = oracle.OracleLevel(sc.domain, sc.nbins)
    for c, dpt in zip(sc.cameras, sc.depths):
        orc.accumulate(c, dpt, 1)
    orc.iterate(sc.iterations)
    Vo, To = oracle.mesh(sc.domain, orc.u.astype(np.float32))
    assert abs(len(V) - len(Vo)) <= 0.01 * len(Vo) and abs(len(T) - len(To)) <= 0.01 * len(To)
    r = np.linalg.norm(V - sc.meta["centre"], axis=1)
    near = np.abs(r - sc.meta["radius"]) < 3 * sc.domain.h
    assert near.mean() > 0.9
    assert np.median(np.abs(r[near] - sc.meta["radius"])) < 0.5 * sc.domain.h
