"""FP64 CPU oracle (test infrastructure) for the histogram + TGV primal-dual path.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference legs are the only users.  The CUDA library never
imports, links or executes anything here, and nothing here imports the CUDA
library: the two share only the seeded inputs of ``synth``.

The arithmetic lives in ``tgv_oracle.c`` (plain loops, FP64; the Alg. 1 bin
decision in FP32 with one rounding per operation).  This module only
marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tgv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

GCC_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile tgv_oracle.c into liboracle.so (gcc, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *GCC_FLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "orc_pyramid_nlevels": (i32, [i32, i32]),
            "orc_pyramid_layout": (i64, [i32, i32, P, P]),
            "orc_build_pyramid": (None, [P, i32, i32, i64, P]),
            "orc_accumulate": (i64, [i64, P, P, f64, f64, P, i32, i32, P, i32, ctypes.c_uint32, P, P]),
            "orc_vote_list": (None, [i64, P, P, f64, f64, P, i32, i32, P, i32, P]),
            "orc_build_links": (i32, [i64, P, i64, P, P, P]),
            "orc_grad": (None, [i64, P, P, P, P]),
            "orc_symgrad": (None, [i64, P, P, P, P]),
            "orc_div1": (None, [i64, P, P, P, P]),
            "orc_div2": (None, [i64, P, P, P, P]),
            "orc_project_p": (None, [i64, P, f64]),
            "orc_project_q": (None, [i64, P, f64]),
            "orc_centre": (f64, [i32, i32, i32]),
            "orc_prox": (f64, [f64, P, i32, f64, f64, i32]),
            "orc_tgv_iterate": (None, [i64, P, P, P, P, P, i32, P, i32, i32, P, P, P, P, P, P, i32, i32]),
            "orc_energy": (None, [i64, P, P, P, P, P, i32, P, i32, f64, P, P, P, P, P]),
            "orc_prolong": (i64, [i64, P, P, P, i64, P, P, P]),
            "orc_max_threads": (i32, []),
            "orc_atan2_as": (ctypes.c_float, [ctypes.c_float, ctypes.c_float]),
            "orc_mesh": (i64, [i64, P, i64, P, P, P, f64, P, P, P]),
            "orc_mc_triangulate": (i32, [i32, P, P, P]),
            "orc_octree_samples": (i64, [P, i32, i32, P, P, f64, i32, i32, P, P, P]),
            "orc_sincos_tay_many": (None, [P, i64, P, P]),
            "orc_octree_build": (i64, [i32, P, i32, i32, P, P, f64, i32, i32, i32, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------- pyramid / Alg. 1
def pyramid_layout(W: int, H: int):
    n = lib().orc_pyramid_nlevels(W, H)
    dims = np.zeros(2 * n, np.int32)
    offs = np.zeros(n, np.int64)
    total = lib().orc_pyramid_layout(W, H, _p(dims), _p(offs))
    return dims.reshape(n, 2), offs, int(total)


def build_pyramid(depth: np.ndarray) -> np.ndarray:
    """All pyramid levels of one depth map, concatenated (float32, NaN = invalid)."""
    d = _c(depth, np.float32)
    H, W = d.shape
    _, _, total = pyramid_layout(W, H)
    out = np.empty(total, np.float32)
    lib().orc_build_pyramid(_p(d), W, H, W, _p(out))
    return out


def pyramid_levels(depth: np.ndarray):
    pyr = build_pyramid(depth)
    H, W = depth.shape
    dims, offs, _ = pyramid_layout(W, H)
    return [pyr[offs[l]: offs[l] + dims[l, 0] * dims[l, 1]].reshape(dims[l, 1], dims[l, 0]) for l in range(len(offs))]


def voxel_radius(desc) -> float:
    r = float(getattr(desc, "radius", 0.0) or 0.0)
    return r if r > 0 else float(desc.h) / 2.0


def mesh(desc, u: np.ndarray):
    """Marching cubes (Sec. 4.6) of the FP32 indicator `u` ((nb + nf) * 512 values:
    active bricks, then frozen) on the level `desc`: (vertices (nv, 3) float32,
    triangles (nt, 3) int32), vertices by increasing edge id, triangles by cell."""
    b = _c(desc.bricks, np.int32).reshape(-1, 3)
    f = _c(desc.frozen, np.int32).reshape(-1, 3) if getattr(desc, "frozen", None) is not None else \
        np.zeros((0, 3), np.int32)
    u32 = _c(u, np.float32).reshape(-1)
    if u32.size != 512 * (b.shape[0] + f.shape[0]):
        raise ValueError("u must hold (nb + nf) * 512 values")
    o = _c(desc.origin, np.float64)
    nv = np.zeros(1, np.int64)
    nt = lib().orc_mesh(b.shape[0], _p(b), f.shape[0], _p(f), _p(u32), _p(o), float(desc.h), _p(nv), None, None)
    if nt < 0:
        raise ValueError("duplicate brick")
    verts = np.zeros((int(nv[0]), 3), np.float32)
    tris = np.zeros((int(nt), 3), np.int32)
    lib().orc_mesh(b.shape[0], _p(b), f.shape[0], _p(f), _p(u32), _p(o), float(desc.h), _p(nv), _p(verts), _p(tris))
    return verts, tris


def triangulate_min_area(P: np.ndarray) -> np.ndarray:
    """The marching-cubes polygon triangulation (FP32 dynamic programming) of the
    polygon P ((k, 3), 3 <= k <= 12): (k - 2, 3) polygon-local vertex indices."""
    P32 = _c(P, np.float32).reshape(-1, 3)
    out = np.zeros((max(1, P32.shape[0] - 2), 3), np.int32)
    n = lib().orc_mc_triangulate(P32.shape[0], _p(P32), None, _p(out))
    return out[:n]


def sincos_tay(x) -> tuple:
    """(sin x, cos x) in FP32 by the oracle's own reduction and Taylor polynomials
    (the spherical unprojection of the octree build), |x| <= 4."""
    x = _c(np.atleast_1d(x), np.float32)
    s = np.empty_like(x)
    c = np.empty_like(x)
    lib().orc_sincos_tay_many(_p(x), x.size, _p(s), _p(c))
    return s, c


def octree_samples(cam, depth: np.ndarray, root_min, root_edge: float, dmin: int, dmax: int):
    """Per pixel of one map (pinhole or spherical): (depth d or -1, cube coords (H, W, 3),
    radius r)."""
    d = _c(depth, np.float32)
    H, W = d.shape
    dd = np.empty((H, W), np.int32)
    qq = np.zeros((H, W, 3), np.int64)
    rr = np.zeros((H, W), np.float32)
    lib().orc_octree_samples(_p(_c(cam.as_array(), np.float64)), W, H, _p(d), _p(_c(root_min, np.float64)),
                             float(root_edge), int(dmin), int(dmax), _p(dd), _p(qq), _p(rr))
    return dd, qq, rr


def octree_build(cams, depths, root_min, root_edge: float, dmin: int, dmax: int, band: int = 1):
    """Brick domain from depth maps (pinhole or spherical; Eq. 4, Sec. 4.1-4.2): per level (active, frozen)
    brick coordinate arrays in Morton order, and the sample count."""
    dep = _c(np.stack(depths), np.float32)
    nm, H, W = dep.shape
    cam = _c(np.stack([c.as_array() for c in cams]), np.float64)
    nlev = dmax - dmin + 1
    counts = np.zeros(2 * nlev, np.int64)
    rm = _c(root_min, np.float64)
    lib().orc_octree_build(nm, _p(cam), W, H, _p(dep), _p(rm), float(root_edge), dmin, dmax, band, _p(counts), None)
    out = np.zeros(3 * int(counts.sum()) + 3, np.int32)
    ns = lib().orc_octree_build(nm, _p(cam), W, H, _p(dep), _p(rm), float(root_edge), dmin, dmax, band, _p(counts),
                                _p(out))
    levels, o = [], 0
    for l in range(nlev):
        a, f = int(counts[2 * l]), int(counts[2 * l + 1])
        levels.append((out[3 * o:3 * (o + a)].reshape(-1, 3).copy(), out[3 * (o + a):3 * (o + a + f)].reshape(-1, 3).copy()))
        o += a + f
    return levels, int(ns)


def prox_many(ut: np.ndarray, hist: np.ndarray, tau: float, lam: float, centres: int = 0) -> np.ndarray:
    """The histogram prox of many voxels at once (T7 read from Eq. 2's data term): the
    median of the 2n + 1 values {c_b} and {ut - tau lam W_i}, W_i = sum_{b<i} h_b - sum_{b>=i} h_b."""
    h = np.asarray(hist, np.float64)
    n = h.shape[1]
    b = np.arange(n)
    c = -1.0 + 2.0 * b / (n - 1) if centres == 0 else -1.0 + (2.0 * b + 1.0) / n
    cum = np.concatenate([np.zeros((h.shape[0], 1)), np.cumsum(h, 1)], 1)  # sum_{b<i}
    W = cum - (cum[:, -1:] - cum)                                            # i = 0..n
    vals = np.concatenate([np.broadcast_to(c, h.shape), ut[:, None] - tau * lam * W], 1)
    return np.median(vals, axis=1)


def atan2_as(y: float, x: float) -> float:
    """The FP32 arctangent of the spherical projection (A&S 4.4.49, explicit rounding)."""
    return float(lib().orc_atan2_as(float(y), float(x)))


def vote_list(idx3: np.ndarray, origin, h: float, r: float, cam, depth: np.ndarray, nbins: int) -> np.ndarray:
    """Alg. 1 decision for a list of global voxel indices: bin, or -1 for no vote."""
    idx3 = _c(idx3, np.int64).reshape(-1, 3)
    pyr = build_pyramid(depth)
    H, W = depth.shape
    out = np.empty(idx3.shape[0], np.int32)
    lib().orc_vote_list(idx3.shape[0], _p(idx3), _p(_c(origin, np.float64)), float(h), float(r),
                        _p(_c(cam.as_array(), np.float64)), W, H, _p(pyr), nbins, _p(out))
    return out


# ----------------------------------------------------------------------------- operators
def links(bricks: np.ndarray, frozen: Optional[np.ndarray] = None):
    b = _c(bricks, np.int32).reshape(-1, 3)
    f = _c(frozen, np.int32).reshape(-1, 3) if frozen is not None else np.zeros((0, 3), np.int32)
    n = 512 * b.shape[0]
    fwd = np.empty(3 * n, np.int64)
    bwd = np.empty(3 * n, np.int64)
    rc = lib().orc_build_links(b.shape[0], _p(b), f.shape[0], _p(f), _p(fwd), _p(bwd))
    if rc != 0:
        raise ValueError("duplicate brick coordinates")
    return fwd, bwd


def grad(fwd, u, fu):
    n = u.shape[0]
    g = np.empty(3 * n)
    lib().orc_grad(n, _p(fwd), _p(_c(u, np.float64)), _p(_c(fu, np.float64)), _p(g))
    return g.reshape(n, 3)


def symgrad(bwd, v, fv):
    v = _c(v, np.float64).reshape(-1, 3)
    n = v.shape[0]
    e = np.empty(6 * n)
    lib().orc_symgrad(n, _p(bwd), _p(v), _p(_c(fv, np.float64)), _p(e))
    return e.reshape(n, 6)


def div1(fwd, bwd, p):
    p = _c(p, np.float64).reshape(-1, 3)
    n = p.shape[0]
    d = np.empty(n)
    lib().orc_div1(n, _p(fwd), _p(bwd), _p(p), _p(d))
    return d


def div2(fwd, bwd, q):
    q = _c(q, np.float64).reshape(-1, 6)
    n = q.shape[0]
    w = np.empty(3 * n)
    lib().orc_div2(n, _p(fwd), _p(bwd), _p(q), _p(w))
    return w.reshape(n, 3)


def project_p(p, alpha1):
    p = np.array(p, dtype=np.float64).reshape(-1, 3)
    lib().orc_project_p(p.shape[0], _p(p), float(alpha1))
    return p


def project_q(q, alpha0):
    q = np.array(q, dtype=np.float64).reshape(-1, 6)
    lib().orc_project_q(q.shape[0], _p(q), float(alpha0))
    return q


def centre(b: int, n: int, centres: int = 0) -> float:
    return lib().orc_centre(b, n, centres)


def prox(ut: float, hb, tau: float, lam: float, centres: int = 0) -> float:
    hb = _c(hb, np.uint32)
    return lib().orc_prox(float(ut), _p(hb), hb.shape[0], float(tau), float(lam), centres)


# ----------------------------------------------------------------------------- a domain level
class OracleLevel:
    """One brick level in FP64: histograms, links, TGV state (u, ubar, v, vbar, p, q).

    Voxel order: brick b of the active list, then local index x + 8y + 64z.
    """

    def __init__(self, desc, nbins: int, alpha1=1.0, alpha0=2.0, lam=1.0, tau=0.2, sigma=0.2,
                 clamp_u=True, centres=0, box_v=2.0):
        self.desc = desc
        self.nbins = int(nbins)
        self.prm = np.array([alpha1, alpha0, lam, tau, sigma], np.float64)
        self.clamp_u = bool(clamp_u)
        self.centres = int(centres)
        self.box_v = float(box_v)
        self.bricks = _c(desc.bricks, np.int32).reshape(-1, 3)
        self.n = 512 * self.bricks.shape[0]
        self.fwd, self.bwd = links(self.bricks, getattr(desc, "frozen", None))
        nf = 0 if getattr(desc, "frozen", None) is None else int(np.asarray(desc.frozen).shape[0])
        self.fu = np.zeros(max(1, 512 * nf))
        self.fv = np.zeros(max(1, 3 * 512 * nf))
        if nf and getattr(desc, "frozen_u", None) is not None:
            self.fu[:512 * nf] = np.asarray(desc.frozen_u, np.float64).reshape(-1)
        if nf and getattr(desc, "frozen_v", None) is not None:
            fv = np.asarray(desc.frozen_v, np.float64).reshape(nf, 3, 512).transpose(0, 2, 1)
            self.fv[:3 * 512 * nf] = fv.reshape(-1)
        self.hist = np.zeros((self.n, self.nbins), np.uint32)
        self.reset()

    def reset(self):
        n = self.n
        self.u = np.zeros(n)
        self.ubar = np.zeros(n)
        self.v = np.zeros((n, 3))
        self.vbar = np.zeros((n, 3))
        self.p = np.zeros((n, 3))
        self.q = np.zeros((n, 6))

    # Alg. 1 over every voxel, one map
    def accumulate(self, cam, depth: np.ndarray, vote: int = 1, diag: bool = False):
        pyr = build_pyramid(depth)
        H, W = depth.shape
        nd = np.zeros(1, np.int64)
        votes = lib().orc_accumulate(self.bricks.shape[0], _p(self.bricks), _p(_c(self.desc.origin, np.float64)),
                                     float(self.desc.h), voxel_radius(self.desc),
                                     _p(_c(cam.as_array(), np.float64)), W, H, _p(pyr), self.nbins,
                                     int(vote), _p(self.hist), _p(nd) if diag else None)
        return (int(votes), int(nd[0])) if diag else int(votes)

    def iterate(self, iters: int, nthreads: int = 0):
        lib().orc_tgv_iterate(self.n, _p(self.fwd), _p(self.bwd), _p(self.fu), _p(self.fv), _p(self.hist),
                              self.nbins, _p(self.prm), int(self.clamp_u), self.centres, _p(self.u), _p(self.ubar),
                              _p(self.v), _p(self.vbar), _p(self.p), _p(self.q), int(iters), int(nthreads))

    def energy(self):
        """(E, D, gap, certified) as in Eq. 2 with the dual of the bounded problem."""
        out = np.zeros(4)
        lib().orc_energy(self.n, _p(self.fwd), _p(self.bwd), _p(self.fu), _p(self.fv), _p(self.hist), self.nbins,
                         _p(self.prm), self.centres, self.box_v, _p(self.u), _p(self.v), _p(self.p), _p(self.q),
                         _p(out))
        return out

    def global_voxels(self) -> np.ndarray:
        li = np.arange(512)
        loc = np.stack([li % 8, (li // 8) % 8, li // 64], axis=1)
        return (8 * self.bricks[:, None, :] + loc[None, :, :]).reshape(-1, 3)

    def prolong_from(self, coarse: "OracleLevel"):
        """Coarse-to-fine start: u from the parent voxel, v halved, duals zero."""
        fine = _c(self.global_voxels(), np.int64)
        fu = np.empty(self.n)
        fv = np.empty(3 * self.n)
        missing = lib().orc_prolong(coarse.bricks.shape[0], _p(coarse.bricks), _p(coarse.u),
                                    _p(_c(coarse.v, np.float64)), self.n, _p(fine), _p(fu), _p(fv))
        self.reset()
        self.u[:] = fu
        self.ubar[:] = fu
        self.v[:] = fv.reshape(-1, 3)
        self.vbar[:] = self.v
        return int(missing)


def prolong_frozen(fine: OracleLevel, coarse: OracleLevel) -> int:
    """Frozen voxels of `fine` take u from their parent voxel on `coarse` and v halved (Sec. 4.5)."""
    fr = getattr(fine.desc, "frozen", None)
    if fr is None or len(fr) == 0:
        return 0
    fr = _c(fr, np.int32).reshape(-1, 3)
    li = np.arange(512)
    loc = np.stack([li % 8, (li // 8) % 8, li // 64], axis=1)
    g = _c((8 * fr[:, None, :] + loc[None]).reshape(-1, 3), np.int64)
    n = g.shape[0]
    fu = np.empty(n)
    fv = np.empty(3 * n)
    missing = lib().orc_prolong(coarse.bricks.shape[0], _p(coarse.bricks), _p(coarse.u),
                                _p(_c(coarse.v, np.float64)), n, _p(g), _p(fu), _p(fv))
    fine.fu[:n] = fu
    fine.fv[:3 * n] = fv
    return int(missing)


def max_threads() -> int:
    return int(lib().orc_max_threads())
