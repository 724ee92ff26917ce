"""Pins of the oracle's TGV operators, prox, projections, energy/gap and iteration.

What fixes each expected value (never the oracle itself):
* adjoint identities <grad u, p> = -<u, div1 p>, <E v, q>_F = -<v, div2 q> (linear algebra);
* an affine field has E(v) = 0 and grad u - v = 0 wherever a forward neighbour exists,
  so its TGV energy is a closed-form sum over the upper boundary faces (Eq. 2-3);
* the prox of the histogram data term, minimised piece by piece (a quadratic on each
  interval between bin centres), plus a dense grid scan;
* weak duality (gap >= 0) and strong duality (gap -> 0 on a small problem);
* the sphere's radius, seen through the whole pipeline (Alg. 1 + Eq. 2 minimisation).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from tests._geom import dense_from_bricks, edge_crossings


def _box(nb):
    return synth.dense_bricks(nb)


def _domains(rng):
    full = synth.DomainDesc(np.zeros(3), 1.0, _box(2))
    holes_b = _box(3)
    holes_b = holes_b[[i for i in range(len(holes_b)) if i not in (4, 13, 20)]]
    holes = synth.DomainDesc(np.zeros(3), 1.0, holes_b)
    act = _box(2)
    shell = np.array([c for c in itertools.product(range(-1, 3), repeat=3)
                      if not all(0 <= x < 2 for x in c) and sum(1 for x in c if 0 <= x < 2) == 2], np.int32)
    frz = synth.DomainDesc(np.zeros(3), 1.0, act, frozen=shell)
    return {"full": full, "holes": holes, "frozen": frz}


@pytest.mark.parametrize("kind", ["full", "holes", "frozen"])
def test_adjoint_identities(kind):
    rng = np.random.default_rng(7)
    dom = _domains(rng)[kind]
    fwd, bwd = oracle.links(dom.bricks, dom.frozen)
    n = 512 * dom.nbricks
    if kind == "full":
        assert (fwd == -1).sum() == 3 * 16 * 16 and (fwd >= 0).sum() == 3 * n - 3 * 256
    if kind == "frozen":
        assert (fwd <= -2).sum() == 3 * 256 and (fwd == -1).sum() == 0
    nf = 512 * dom.nfrozen
    fu0, fv0 = np.zeros(max(1, nf)), np.zeros(max(1, 3 * nf))
    u = rng.standard_normal(n)
    p = rng.standard_normal((n, 3))
    v = rng.standard_normal((n, 3))
    q = rng.standard_normal((n, 6))
    g = oracle.grad(fwd, u, fu0)
    lhs = np.sum(g * p)
    rhs = -np.sum(u * oracle.div1(fwd, bwd, p))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    e = oracle.symgrad(bwd, v, fv0)
    w = np.array([1, 1, 1, 2, 2, 2.0])  # Frobenius: off-diagonal pairs count twice
    lhs = np.sum(e * q * w)
    rhs = -np.sum(v * oracle.div2(fwd, bwd, q))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def _affine_box(nb, gvec, b0):
    dom = synth.DomainDesc(np.zeros(3), 1.0, _box(nb))
    lvl = oracle.OracleLevel(dom, 8)
    x = lvl.global_voxels().astype(np.float64)
    u = x @ gvec + b0
    return dom, lvl, u


def test_affine_field_energy_closed_form():
    gvec = np.array([0.011, -0.007, 0.005])
    nb = 2
    N = 8 * nb
    dom, lvl, u = _affine_box(nb, gvec, -0.1)
    lvl.u[:] = u
    lvl.v[:] = gvec[None, :]
    E, D, gap, cert = lvl.energy()  # zero histograms: no data term
    # voxels on the upper faces lack the forward link on those axes: there grad u - v = -g_a
    want = 0.0
    for S in itertools.chain.from_iterable(itertools.combinations(range(3), k) for k in range(4)):
        count = (N - 1) ** (3 - len(S))
        want += count * math.sqrt(sum(gvec[a] ** 2 for a in S))
    assert abs(E - 1.0 * want) <= 1e-12 * want
    # and E(v) = 0 for a constant v (alpha0 term vanishes): perturbing alpha0 changes nothing
    lvl.prm[1] = 123.0
    assert abs(lvl.energy()[0] - E) <= 1e-12 * E


def test_affine_field_is_stationary_in_the_interior():
    gvec = np.array([0.02, 0.01, -0.015])
    dom, lvl, u = _affine_box(3, gvec, 0.05)
    lvl.u[:] = u
    lvl.ubar[:] = u
    lvl.v[:] = gvec
    lvl.vbar[:] = gvec
    k = 3
    lvl.iterate(k)
    x = lvl.global_voxels()
    N = 24
    # the boundary disturbance travels at most two voxels per iteration
    interior = np.all((x >= 2 * k + 2) & (x < N - 2 * k - 2), axis=1)
    assert interior.sum() > 500
    assert np.max(np.abs(lvl.u[interior] - u[interior])) <= 1e-12
    assert np.max(np.abs(lvl.v[interior] - gvec)) <= 1e-12
    assert np.max(np.abs(lvl.p[interior])) <= 1e-12 and np.max(np.abs(lvl.q[interior])) <= 1e-12


def test_frozen_halo_with_affine_values_keeps_a_chunk_exact():
    """FRZ links act as neighbours with fixed u, v: an affine chunk inside an affine frozen
    shell has no boundary at all, so every voxel keeps its state and E = 0 exactly.
    Dyadic slopes make every value exact in float32 and float64."""
    gvec = np.array([1 / 64, -1 / 128, 1 / 32])
    act = _box(2)
    shell = np.array([c for c in itertools.product(range(-1, 3), repeat=3)
                      if not all(0 <= x < 2 for x in c) and sum(1 for x in c if 0 <= x < 2) == 2], np.int32)
    li = np.arange(512)
    loc = np.stack([li % 8, (li // 8) % 8, li // 64], axis=1)
    fx = (8 * shell[:, None, :] + loc[None]).astype(np.float64)
    fu = (fx @ gvec - 0.125).astype(np.float32)
    fvv = np.broadcast_to(gvec.astype(np.float32)[None, :, None], (len(shell), 3, 512)).copy()
    dom = synth.DomainDesc(np.zeros(3), 1.0, act, frozen=shell, frozen_u=fu, frozen_v=fvv)
    lvl = oracle.OracleLevel(dom, 8)
    ua = lvl.global_voxels().astype(np.float64) @ gvec - 0.125
    assert np.all(np.abs(ua) <= 1.0)
    lvl.u[:] = ua
    lvl.ubar[:] = ua
    lvl.v[:] = gvec
    lvl.vbar[:] = gvec
    assert lvl.energy()[0] == 0.0
    lvl.iterate(5)
    np.testing.assert_array_equal(lvl.u, ua)
    np.testing.assert_array_equal(lvl.v, np.broadcast_to(gvec, lvl.v.shape))
    assert np.all(lvl.p == 0) and np.all(lvl.q == 0)
    # the same chunk with the shell removed (NONE links) is not stationary
    lvl2 = oracle.OracleLevel(synth.DomainDesc(np.zeros(3), 1.0, act), 8)
    lvl2.u[:] = ua
    lvl2.ubar[:] = ua
    lvl2.v[:] = gvec
    lvl2.vbar[:] = gvec
    assert lvl2.energy()[0] > 0.0
    lvl2.iterate(5)
    assert np.max(np.abs(lvl2.u - ua)) > 1e-4


def _prox_piecewise(ut, hb, tau, lam, centres):
    """Exact argmin of (u-ut)^2/(2 tau) + lam sum_b h_b |u - c_b|, one quadratic piece at a time."""
    n = len(hb)
    c = [(-1 + 2 * b / (n - 1)) if centres == 0 else (-1 + (2 * b + 1) / n) for b in range(n)]

    def f(u):
        return (u - ut) ** 2 / (2 * tau) + lam * sum(h * abs(u - cb) for h, cb in zip(hb, c))

    cands = []
    for i in range(n + 1):
        lo = -math.inf if i == 0 else c[i - 1]
        hi = math.inf if i == n else c[i]
        slope = sum(hb[b] for b in range(i)) - sum(hb[b] for b in range(i, n))
        cands.append(min(max(ut - tau * lam * slope, lo), hi))
    best = min(cands, key=f)
    return best, f


@pytest.mark.parametrize("centres", [0, 1])
def test_prox_matches_piecewise_minimum_and_grid(centres):
    rng = np.random.default_rng(11)
    for trial in range(400):
        n = int(rng.integers(2, 5))
        hb = rng.integers(0, 6, size=n).astype(np.uint32)
        ut = float(rng.uniform(-3, 3))
        tau = float(rng.choice([0.2, 0.05, 1.0]))
        lam = float(rng.choice([1.0, 0.3]))
        got = oracle.prox(ut, hb, tau, lam, centres)
        want, f = _prox_piecewise(ut, [int(x) for x in hb], tau, lam, centres)
        assert abs(got - want) <= 1e-12, (trial, n, hb, ut)
        if trial < 40:
            grid = np.arange(-8.0, 8.0, 1e-4)
            fg = (grid - ut) ** 2 / (2 * tau) + lam * sum(
                int(h) * np.abs(grid - oracle.centre(b, n, centres)) for b, h in enumerate(hb))
            assert f(got) <= fg.min() + 1e-12


def test_prox_empty_histogram_is_identity():
    for ut in (-2.5, -0.3, 0.0, 0.7, 4.0):
        assert oracle.prox(ut, np.zeros(8, np.uint32), 0.2, 1.0) == ut


def test_bin_centres():
    assert [oracle.centre(b, 8, 0) for b in (0, 7)] == [-1.0, 1.0]
    assert abs(oracle.centre(3, 8, 0) - (-1 + 6 / 7)) < 1e-15
    assert [oracle.centre(b, 4, 1) for b in range(4)] == [-0.75, -0.25, 0.25, 0.75]


def test_projections_idempotent_nonexpansive():
    rng = np.random.default_rng(3)
    p = rng.standard_normal((500, 3)) * 2
    q = rng.standard_normal((500, 6)) * 3
    a1, a0 = 1.0, 2.0
    P = oracle.project_p(p, a1)
    Q = oracle.project_q(q, a0)
    fro = lambda m: np.sqrt(m[:, 0] ** 2 + m[:, 1] ** 2 + m[:, 2] ** 2 + 2 * (m[:, 3] ** 2 + m[:, 4] ** 2 + m[:, 5] ** 2))
    assert np.all(np.linalg.norm(P, axis=1) <= a1 * (1 + 1e-14))
    assert np.all(fro(Q) <= a0 * (1 + 1e-14))
    # idempotent up to one rounding of the norm
    np.testing.assert_allclose(oracle.project_p(P, a1), P, rtol=1e-15, atol=0)
    np.testing.assert_allclose(oracle.project_q(Q, a0), Q, rtol=1e-15, atol=0)
    inside = np.linalg.norm(p, axis=1) <= a1
    np.testing.assert_array_equal(P[inside], p[inside])
    # non-expansive (in the Frobenius metric for q)
    p2 = p + rng.standard_normal(p.shape) * 0.3
    q2 = q + rng.standard_normal(q.shape) * 0.3
    P2, Q2 = oracle.project_p(p2, a1), oracle.project_q(q2, a0)
    assert np.all(np.linalg.norm(P - P2, axis=1) <= np.linalg.norm(p - p2, axis=1) + 1e-14)
    assert np.all(fro(Q - Q2) <= fro(q - q2) + 1e-14)
    # the projection is the nearest point: radial scaling of p onto the sphere
    out = ~inside
    np.testing.assert_allclose(P[out], p[out] / np.linalg.norm(p[out], axis=1, keepdims=True), rtol=1e-15)


def test_gap_nonnegative_and_vanishes_on_small_problem():
    rng = np.random.default_rng(5)
    dom = synth.DomainDesc(np.zeros(3), 1.0, _box(1))
    lvl = oracle.OracleLevel(dom, 6)
    lvl.hist[:] = synth.random_histograms(rng, lvl.n, 6, max_count=3)
    gaps = []
    for k in range(60):
        lvl.iterate(50)
        E, D, gap, cert = lvl.energy()
        assert cert == 1.0
        assert gap >= -1e-9 * abs(E)
        gaps.append(gap / E)
    # strong duality: the relative gap keeps shrinking (about 4e-6 after 3000 iterations)
    assert gaps[-1] < 1e-5 and gaps[-1] < 0.01 * gaps[0], (gaps[0], gaps[-1])


def test_frozen_domain_gap_nonnegative():
    rng = np.random.default_rng(9)
    specs = synth.chunk_workload(seed=99, nchunks=1, min_vox=4096, max_vox=4096, nbins_range=(8, 8))
    sp = specs[0]
    lvl = oracle.OracleLevel(sp.domain, sp.nbins)
    lvl.hist[:] = sp.hist
    for k in range(8):
        lvl.iterate(25)
        E, D, gap, cert = lvl.energy()
        assert cert == 1.0 and gap >= -1e-9 * abs(E)
    assert rng is not None


def test_thread_count_does_not_change_iterates():
    rng = np.random.default_rng(1)
    dom = synth.DomainDesc(np.zeros(3), 1.0, _box(2))
    a = oracle.OracleLevel(dom, 8)
    a.hist[:] = synth.random_histograms(rng, a.n, 8)
    b = oracle.OracleLevel(dom, 8)
    b.hist[:] = a.hist
    a.iterate(20, nthreads=1)
    b.iterate(20, nthreads=4)
    for f in ("u", "ubar", "v", "vbar", "p", "q"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_prolongation_by_hand():
    coarse = synth.DomainDesc(np.zeros(3), 1.0, np.array([[0, 0, 0]], np.int32))
    fine = synth.DomainDesc(np.zeros(3), 0.5, np.array([[1, 0, 0], [0, 1, 1]], np.int32))
    c = oracle.OracleLevel(coarse, 8)
    c.u[:] = np.arange(512) / 512.0
    c.v[:] = np.arange(1536).reshape(512, 3)
    f = oracle.OracleLevel(fine, 8)
    assert f.prolong_from(c) == 0
    # fine voxel (8+i, j, k) of brick (1,0,0) has parent coarse voxel (4 + i//2, j//2, k//2)
    for (i, j, k) in [(0, 0, 0), (1, 1, 1), (7, 3, 6)]:
        fi = 0 * 512 + i + 8 * j + 64 * k
        ci = (4 + i // 2) + 8 * (j // 2) + 64 * (k // 2)
        assert f.u[fi] == c.u[ci] and f.ubar[fi] == c.u[ci]
        np.testing.assert_array_equal(f.v[fi], 0.5 * c.v[ci])
    # brick (0,1,1): fine (i, 8+j, 8+k) -> coarse (i//2, 4 + j//2, 4 + k//2)
    fi = 512 + 5 + 8 * 2 + 64 * 7
    ci = 2 + 8 * (4 + 1) + 64 * (4 + 3)
    assert f.u[fi] == c.u[ci]
    assert np.all(f.p == 0) and np.all(f.q == 0)


@pytest.fixture(scope="module")
def sphere_run():
    sc = synth.sphere_scene()
    lvl = oracle.OracleLevel(sc.domain, sc.nbins)
    for cam, d in zip(sc.cameras, sc.depths):
        lvl.accumulate(cam, d, 1)
    trace = []
    for k in range(sc.iterations // 25):
        lvl.iterate(25)
        trace.append(lvl.energy())
    return sc, lvl, np.array(trace)


def test_sphere_gap_certified_nonnegative_and_decreasing(sphere_run):
    sc, lvl, tr = sphere_run
    assert np.all(tr[:, 3] == 1.0)
    assert np.all(tr[:, 2] >= 0.0)
    # empirical on this scene: the gap at every 25-iteration checkpoint does not increase
    assert np.all(np.diff(tr[:, 2]) <= 0.0), tr[:, 2]
    assert tr[-1, 2] < 0.15 * tr[0, 2]


def test_sphere_zero_level_set_matches_radius(sphere_run):
    sc, lvl, _ = sphere_run
    n = 64
    U = dense_from_bricks(lvl.u, sc.domain.bricks, n)
    seen = dense_from_bricks(lvl.hist.sum(axis=1), sc.domain.bricks, n) >= 2
    pos, _ = edge_crossings(U, seen, sc.domain.h)
    err = (np.linalg.norm(pos - 0.5, axis=1) - 0.35) / sc.domain.h
    assert len(err) > 5000
    a = np.abs(err)
    # reading of the tolerance: mean within 0.5 h, 99% within 1 h, all within 1.5 h
    assert a.mean() <= 0.5 and np.percentile(a, 99) <= 1.0 and a.max() <= 1.5, (a.mean(), a.max())
