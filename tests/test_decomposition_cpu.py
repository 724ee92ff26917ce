"""One domain split across ranks (the multi-GPU design for a level larger than one GPU):
z-slabs with one halo exchange per half-step -- ubar and vbar faces before the dual step,
the new p and q faces before the primal step -- over 2 and 4 gloo ranks on CPU.

The iteration (Eq. 2-3 with the primal-dual steps of Sec. 3.2) is written here once, in
FP64 numpy on slabs with ghost layers; the split run equals the unsplit run bit for bit,
and the unsplit run equals the C oracle's iteration of the same level to 1e-10.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth

NB = 3          # bricks per axis: a 24^3 voxel box
NBINS = 8
ITERS = 20
TAU = SIGMA = 0.2
ALPHA1, ALPHA0, LAM = 1.0, 2.0, 1.0


def problem():
    rng = np.random.default_rng(17)
    n = 8 * NB
    hist = rng.integers(0, 9, size=(n, n, n, NBINS)).astype(np.float64)  # (z, y, x, bin)
    return hist


def fwd_diff(a, axis, has_hi):
    """Forward difference of the owned layers (ghost layers 0 and -1 along z, axis 0)."""
    if axis == 0:
        d = a[2:] - a[1:-1]
        if not has_hi:
            d[-1] = 0.0
        return d
    o = a[1:-1]
    d = np.zeros_like(o)
    sl_hi = [slice(None)] * 3
    sl_lo = [slice(None)] * 3
    sl_hi[axis] = slice(1, None)
    sl_lo[axis] = slice(0, -1)
    d[tuple(sl_lo)] = o[tuple(sl_hi)] - o[tuple(sl_lo)]
    return d


def bwd_diff(a, axis, has_lo):
    if axis == 0:
        d = a[1:-1] - a[:-2]
        if not has_lo:
            d[0] = 0.0
        return d
    o = a[1:-1]
    d = np.zeros_like(o)
    sl_hi = [slice(None)] * 3
    sl_lo = [slice(None)] * 3
    sl_hi[axis] = slice(1, None)
    sl_lo[axis] = slice(0, -1)
    d[tuple(sl_hi)] = o[tuple(sl_hi)] - o[tuple(sl_lo)]
    return d


def dual_step(S, has_lo, has_hi):
    """p, q of the owned layers from ubar, vbar (their ghost layers filled)."""
    # numpy axis 0 = z, 1 = y, 2 = x; component order x, y, z
    ax = [2, 1, 0]
    g = [fwd_diff(S["ub"], ax[a], has_hi) for a in range(3)]
    dm = [[bwd_diff(S["vb"][c], ax[a], has_lo) for c in range(3)] for a in range(3)]
    p = [S["p"][c][1:-1] + SIGMA * (g[c] - S["vb"][c][1:-1]) for c in range(3)]
    n = np.sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2])
    s = np.maximum(1.0, n / ALPHA1)
    for c in range(3):
        S["p"][c][1:-1] = p[c] / s
    e = [dm[0][0], dm[1][1], dm[2][2], 0.5 * (dm[0][1] + dm[1][0]), 0.5 * (dm[0][2] + dm[2][0]),
         0.5 * (dm[1][2] + dm[2][1])]
    q = [S["q"][c][1:-1] + SIGMA * e[c] for c in range(6)]
    n = np.sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + 2.0 * (q[3] * q[3] + q[4] * q[4] + q[5] * q[5]))
    s = np.maximum(1.0, n / ALPHA0)
    for c in range(6):
        S["q"][c][1:-1] = q[c] / s


QIDX = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]


def primal_step(S, has_lo, has_hi):
    """u, v, ubar, vbar of the owned layers from the new p, q (their ghost layers filled)."""
    ax = [2, 1, 0]
    own = S["u"].shape[0] - 2
    d1 = np.zeros_like(S["u"][1:-1])
    for a in range(3):
        # [fwd exists] p_a(y) - [bwd exists] p_a(y - e_a)
        pa = S["p"][a]
        fwd_ok = np.ones_like(d1, bool)
        bwd_ok = np.ones_like(d1, bool)
        sl = [slice(None)] * 3
        if ax[a] == 0:
            if not has_hi:
                fwd_ok[-1] = False
            if not has_lo:
                bwd_ok[0] = False
            back = pa[:-2]
        else:
            sl[ax[a]] = -1
            fwd_ok[tuple(sl)] = False
            sl[ax[a]] = 0
            bwd_ok[tuple(sl)] = False
            back = np.roll(pa[1:-1], 1, axis=ax[a])
        d1 = d1 + np.where(fwd_ok, pa[1:-1], 0.0) - np.where(bwd_ok, back, 0.0)
    d2 = [np.zeros_like(d1) for _ in range(3)]
    for a in range(3):
        fwd_ok = np.ones_like(d1, bool)
        bwd_ok = np.ones_like(d1, bool)
        sl = [slice(None)] * 3
        if ax[a] == 0:
            if not has_hi:
                fwd_ok[-1] = False
            if not has_lo:
                bwd_ok[0] = False
        else:
            sl[ax[a]] = -1
            fwd_ok[tuple(sl)] = False
            sl[ax[a]] = 0
            bwd_ok[tuple(sl)] = False
        for b in range(3):
            qab = S["q"][QIDX[a][b]]
            nxt = qab[2:] if ax[a] == 0 else np.roll(qab[1:-1], -1, axis=ax[a])
            d2[b] = d2[b] + np.where(fwd_ok, nxt, 0.0) - np.where(bwd_ok, qab[1:-1], 0.0)
    u0 = S["u"][1:-1].copy()
    ut = u0 + TAU * d1
    h = S["hist"].reshape(-1, NBINS)
    un = np.clip(oracle.prox_many(ut.reshape(-1), h, TAU, LAM), -1.0, 1.0).reshape(ut.shape)
    S["u"][1:-1] = un
    S["ub"][1:-1] = 2.0 * un - u0
    for c in range(3):
        v0 = S["v"][c][1:-1].copy()
        v1 = v0 + TAU * (S["p"][c][1:-1] + d2[c])
        S["v"][c][1:-1] = v1
        S["vb"][c][1:-1] = 2.0 * v1 - v0
    assert own == un.shape[0]


def new_state(hist_slab):
    nz, ny, nx = hist_slab.shape[:3]
    z = lambda: np.zeros((nz + 2, ny, nx))
    return dict(u=z(), ub=z(), v=[z() for _ in range(3)], vb=[z() for _ in range(3)], p=[z() for _ in range(3)],
                q=[z() for _ in range(6)], hist=hist_slab)


def run_unsplit(hist):
    S = new_state(hist)
    for _ in range(ITERS):
        dual_step(S, False, False)
        primal_step(S, False, False)
    return S["u"][1:-1]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    hist = problem()
    n = hist.shape[0]
    z0, z1 = rank * n // world, (rank + 1) * n // world
    has_lo, has_hi = rank > 0, rank < world - 1
    S = new_state(hist[z0:z1])

    def exchange(up_fields, down_fields):
        """up_fields: the next rank needs my last owned layer (its ghost 0); down_fields: the
        previous rank needs my first owned layer (its ghost -1)."""
        reqs, recv, keep = [], [], []  # keep: send buffers alive until the waits
        for f in up_fields:
            if has_hi:
                keep.append(torch.from_numpy(np.ascontiguousarray(f[-2])))
                reqs.append(dist.isend(keep[-1], rank + 1))
            if has_lo:
                t = torch.empty(f.shape[1:], dtype=torch.float64)
                reqs.append(dist.irecv(t, rank - 1))
                recv.append((f, 0, t))
        for f in down_fields:
            if has_lo:
                keep.append(torch.from_numpy(np.ascontiguousarray(f[1])))
                reqs.append(dist.isend(keep[-1], rank - 1))
            if has_hi:
                t = torch.empty(f.shape[1:], dtype=torch.float64)
                reqs.append(dist.irecv(t, rank + 1))
                recv.append((f, -1, t))
        for r in reqs:
            r.wait()
        for f, k, t in recv:
            f[k] = t.numpy()

    for _ in range(ITERS):
        exchange(up_fields=S["vb"], down_fields=[S["ub"]])   # backward vbar, forward ubar
        dual_step(S, has_lo, has_hi)
        exchange(up_fields=S["p"], down_fields=S["q"])       # backward p (div1), forward q (div2)
        primal_step(S, has_lo, has_hi)
    gathered = [None] * world
    dist.all_gather_object(gathered, (z0, S["u"][1:-1].copy()))
    if rank == 0:
        u = np.zeros((n, n, n))
        for a, part in gathered:
            u[a:a + part.shape[0]] = part
        np.save(os.path.join(out_dir, f"u{world}.npy"), u)
    dist.destroy_process_group()


def test_unsplit_iteration_equals_the_c_oracle():
    hist = problem()
    u = run_unsplit(hist)
    n = 8 * NB
    desc = synth.DomainDesc(np.zeros(3), 1.0, synth.dense_bricks(NB))
    lvl = oracle.OracleLevel(desc, NBINS, alpha1=ALPHA1, alpha0=ALPHA0, lam=LAM, tau=TAU, sigma=SIGMA)
    b = desc.bricks
    loc = np.arange(512)
    g = (8 * b[:, None, :] + np.stack([loc & 7, (loc >> 3) & 7, loc >> 6], 1)[None]).reshape(-1, 3)  # (x, y, z)
    lvl.hist[:] = hist[g[:, 2], g[:, 1], g[:, 0]].astype(np.uint32)
    lvl.iterate(ITERS)
    want = np.zeros((n, n, n))
    want[g[:, 2], g[:, 1], g[:, 0]] = lvl.u
    assert np.abs(u).max() > 0.1
    np.testing.assert_allclose(u, want, rtol=0, atol=1e-10)


@pytest.mark.parametrize("world", [2, 4])
def test_split_with_halo_exchange_equals_unsplit(tmp_path, world):
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = np.load(tmp_path / f"u{world}.npy")
    np.testing.assert_array_equal(got, run_unsplit(problem()))
