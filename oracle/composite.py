"""FP64 oracle of the joint (composite-grid) TGV solve across levels (test infrastructure).

TEST INFRASTRUCTURE ONLY (same users as the rest of ``oracle``).

The paper solves on a 2:1-balanced octree where a cube can have up to four
neighbours over a face (Sec. 3.3) and does not print the operators there.
Reading (stated here and in the library's header):

* levels l = 0..L-1 share the origin, voxel edge halving per level; a voxel of
  level l is a *leaf* when it lies in an active brick of level l and its 8
  children are not in an active brick of level l+1 (children of one voxel lie in
  one finer brick, so they are all present or all absent);
* every difference is a unit index step, as on a single level.  For leaf x and
  axis a, the +a neighbours are: the same-level leaf x + e_a; else, when level
  l has no voxel there, the coarser leaf containing it (one value); else, when
  that voxel is refined, its 4 children on the face next to x (their mean);
  else none.  The -a neighbours likewise;
* forward differences  (G_a u)(x) = mean(u over +a neighbours) - u(x)  (0 if none),
  backward differences (B_a w)(x) = w(x) - mean(w over -a neighbours) (0 if none);
  E(v)_ab = (B_a v_b + B_b v_a) / 2; div1 = -sum_a G_a^T, (div2 q)_b = -sum_a B_a^T q_ab:
  exact negative adjoints, so the primal-dual iteration keeps its convergence
  condition tau sigma ||K||^2 < 1;
* the data term of a leaf uses the histogram of its own level; outer
  boundaries are Neumann (no frozen set).

On a single level the operators reduce to those of ``tgv_oracle.c``
(checked in tests/test_oracle_composite.py).  Leaf order: level by level, then
brick order, then local voxel index.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp



def _voxels(bricks: np.ndarray) -> np.ndarray:
    b = np.asarray(bricks, np.int64).reshape(-1, 3)
    loc = np.arange(512)
    off = np.stack([loc & 7, (loc >> 3) & 7, loc >> 6], 1)
    return (8 * b[:, None, :] + off[None, :, :]).reshape(-1, 3)


class Composite:
    """Leaves, operators and the FP64 iteration of a nested set of brick levels."""

    def __init__(self, level_bricks, nbins: int, alpha1=1.0, alpha0=2.0, lam=1.0, tau=0.2, sigma=0.2,
                 clamp_u=True, centres=0):
        self.nlev = len(level_bricks)
        self.nbins = int(nbins)
        self.alpha1, self.alpha0, self.lam, self.tau, self.sigma = alpha1, alpha0, lam, tau, sigma
        self.clamp_u, self.centres = bool(clamp_u), int(centres)
        vox = [_voxels(b) for b in level_bricks]
        present = [set(map(tuple, v.tolist())) for v in vox]
        self.level_slots = []  # per level: slots (brick * 512 + local) of its leaves
        leaf_keys = []
        for l, v in enumerate(vox):
            finer = present[l + 1] if l + 1 < self.nlev else set()
            keep = [i for i, g in enumerate(v.tolist()) if (2 * g[0], 2 * g[1], 2 * g[2]) not in finer]
            self.level_slots.append(np.array(keep, np.int64))
            leaf_keys += [(l, *tuple(v[i])) for i in keep]
        self.keys = leaf_keys
        self.n = len(leaf_keys)
        index = {k: i for i, k in enumerate(leaf_keys)}
        self.index = index

        def neighbours(l, g, a, s):
            """Leaves next to (l, g) on its s = +1 / -1 side along axis a."""
            q = list(g)
            q[a] += s
            q = tuple(q)
            if (l, *q) in index:
                return [index[(l, *q)]]
            if q in present[l]:  # refined: the 4 children on the face next to g
                out = []
                c0 = [2 * q[0], 2 * q[1], 2 * q[2]]
                if s < 0:
                    c0[a] += 1
                others = [b for b in range(3) if b != a]
                for d0 in (0, 1):
                    for d1 in (0, 1):
                        c = list(c0)
                        c[others[0]] += d0
                        c[others[1]] += d1
                        k = (l + 1, *c)
                        if k not in index:
                            raise ValueError("levels are not 2:1 nested")
                        out.append(index[k])
                return out
            if l > 0:
                k = (l - 1, q[0] >> 1, q[1] >> 1, q[2] >> 1)
                if k in index:
                    return [index[k]]
            return []

        G, B = [], []
        for a in range(3):
            rg, cg, vg, rb, cb, vb = [], [], [], [], [], []
            for i, (l, *g) in enumerate(leaf_keys):
                f = neighbours(l, g, a, +1)
                if f:
                    rg += [i] + [i] * len(f)
                    cg += [i] + f
                    vg += [-1.0] + [1.0 / len(f)] * len(f)
                bk = neighbours(l, g, a, -1)
                if bk:
                    rb += [i] + [i] * len(bk)
                    cb += [i] + bk
                    vb += [1.0] + [-1.0 / len(bk)] * len(bk)
            G.append(sp.csr_matrix((vg, (rg, cg)), shape=(self.n, self.n)))
            B.append(sp.csr_matrix((vb, (rb, cb)), shape=(self.n, self.n)))
        self.G, self.B = G, B
        self.hist = np.zeros((self.n, self.nbins), np.uint32)
        self.leaf_level = np.array([k[0] for k in leaf_keys], np.int64)
        self.reset()

    def reset(self):
        n = self.n
        self.u = np.zeros(n)
        self.ubar = np.zeros(n)
        self.v = np.zeros((n, 3))
        self.vbar = np.zeros((n, 3))
        self.p = np.zeros((n, 3))
        self.q = np.zeros((n, 6))

    def set_level_histograms(self, l: int, hist_level: np.ndarray):
        """hist_level: (nbricks_l * 512, nbins) counts of every voxel of level l."""
        o = int(np.sum([len(s) for s in self.level_slots[:l]]))
        s = self.level_slots[l]
        self.hist[o:o + len(s)] = np.asarray(hist_level)[s]

    def set_level_field(self, l: int, u_level: np.ndarray):
        o = int(np.sum([len(s) for s in self.level_slots[:l]]))
        s = self.level_slots[l]
        self.u[o:o + len(s)] = np.asarray(u_level, np.float64)[s]
        self.ubar[o:o + len(s)] = self.u[o:o + len(s)]

    def level_values(self, l: int):
        o = int(np.sum([len(s) for s in self.level_slots[:l]]))
        return self.level_slots[l], self.u[o:o + len(self.level_slots[l])]

    # --- operators
    def grad(self, u):
        return np.stack([G @ u for G in self.G], 1)

    def symgrad(self, v):
        d = [[self.B[a] @ v[:, b] for b in range(3)] for a in range(3)]
        return np.stack([d[0][0], d[1][1], d[2][2], 0.5 * (d[0][1] + d[1][0]), 0.5 * (d[0][2] + d[2][0]),
                         0.5 * (d[1][2] + d[2][1])], 1)

    def div1(self, p):
        return -sum(self.G[a].T @ p[:, a] for a in range(3))

    QIDX = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]

    def div2(self, q):
        return np.stack([-sum(self.B[a].T @ q[:, self.QIDX[a][b]] for a in range(3)) for b in range(3)], 1)

    def iterate(self, iters: int):
        """Chambolle-Pock (theta = 1) in the step order of the single-level solve."""
        from . import prox_many
        for _ in range(int(iters)):
            p = self.p + self.sigma * (self.grad(self.ubar) - self.vbar)
            n = np.linalg.norm(p, axis=1)
            p /= np.maximum(1.0, n / self.alpha1)[:, None]
            q = self.q + self.sigma * self.symgrad(self.vbar)
            nq = np.sqrt(np.sum(q[:, :3] ** 2, 1) + 2 * np.sum(q[:, 3:] ** 2, 1))
            q /= np.maximum(1.0, nq / self.alpha0)[:, None]
            ut = self.u + self.tau * self.div1(p)
            un = prox_many(ut, self.hist, self.tau, self.lam, self.centres)
            if self.clamp_u:
                un = np.clip(un, -1.0, 1.0)
            vn = self.v + self.tau * (p + self.div2(q))
            self.ubar = 2 * un - self.u
            self.vbar = 2 * vn - self.v
            self.u, self.v, self.p, self.q = un, vn, p, q

    def op_norm2(self, iters: int = 300, seed: int = 0) -> float:
        """||K||^2 for K(u, v) = (grad u - v, E v) (Frobenius pairing on E v): the
        largest eigenvalue of K^T K by power iteration, K^T(g, e) = (-div1 g, -g - div2 e)."""
        rng = np.random.default_rng(seed)
        u = rng.normal(size=self.n)
        v = rng.normal(size=(self.n, 3))
        lam = 0.0
        for _ in range(iters):
            nx = np.sqrt(np.sum(u * u) + np.sum(v * v))
            u, v = u / nx, v / nx
            g = self.grad(u) - v
            e = self.symgrad(v)
            ku = -self.div1(g)
            kv = -g - self.div2(e)
            lam = float(np.sqrt(np.sum(ku * ku) + np.sum(kv * kv)))
            u, v = ku, kv
        return lam


def leaf_keys(level_bricks):
    """(level, x, y, z) of every leaf in the composite order (level, brick, local voxel):
    the voxels of level l whose children are not in an active brick of level l + 1."""
    vox = [_voxels(b) for b in level_bricks]
    keys = []
    for l, v in enumerate(vox):
        finer = set(map(tuple, vox[l + 1].tolist())) if l + 1 < len(vox) else set()
        keys += [(l, *g) for g in v.tolist() if (2 * g[0], 2 * g[1], 2 * g[2]) not in finer]
    return keys


def morton_code(x, y, z, bits: int):
    """Morton code of non-negative integer coordinates: bit b of x, y, z at bits 3b,
    3b + 1, 3b + 2 (one bit at a time, plain integer arithmetic)."""
    x, y, z = (np.asarray(a, np.uint64) for a in (x, y, z))
    m = np.zeros(x.shape, np.uint64)
    one = np.uint64(1)
    for b in range(bits):
        sb = np.uint64(b)
        m |= ((x >> sb) & one) << np.uint64(3 * b)
        m |= ((y >> sb) & one) << np.uint64(3 * b + 1)
        m |= ((z >> sb) & one) << np.uint64(3 * b + 2)
    return m


def treetop(keys, nlev: int, root_bits: int, max_cubes: int):
    """Treetop of the leaf cubes (Sec. 4.3): the smallest rooted subtree of the octree
    whose leaf nodes each hold fewer than max_cubes cubes.

    keys: (level, x, y, z) of every leaf (``Composite.keys``); a leaf of level l is
    the cube of edge 2^(nlev-1-l) at (x, y, z) 2^(nlev-1-l) in finest voxel units.
    The root is [0, 2^root_bits)^3; a node of depth k is an aligned cube of edge
    2^(root_bits - k), its children numbered x + 2 y + 4 z by their half along
    each axis, its code the child numbers from the root down (three bits each).
    A node holds the cubes whose lower corner lies in it.  Nodes with no cube are
    not parts.  Starting from the root, a node holding fewer than max_cubes cubes
    is a part; any other node is split into its children.

    Returns (depth, code, first, last, part): per part in Z-order (Morton order of
    the lower corners), the range [first, last] of the Z-ordered cubes it holds, and
    the part of every leaf (key order).  Raises ValueError when a cube lies outside
    the root or a part's cubes are not consecutive in Z-order."""
    k = np.asarray(keys, np.int64).reshape(-1, 4)
    n = len(k)
    size = np.left_shift(np.int64(1), (nlev - 1 - k[:, 0]))
    corner = k[:, 1:] * size[:, None]
    if n and (corner.min() < 0 or corner.max() >= (1 << root_bits)):
        raise ValueError("a cube lies outside the root")
    z = morton_code(corner[:, 0], corner[:, 1], corner[:, 2], root_bits)
    order = np.argsort(z, kind="stable")
    zpos = np.empty(n, np.int64)
    zpos[order] = np.arange(n)
    parts = []  # (depth, code, first, last)

    def visit(depth, code, lo, members):
        if len(members) == 0:
            return
        if len(members) < max_cubes:
            pos = np.sort(zpos[members])
            if pos[-1] - pos[0] + 1 != len(pos):
                raise ValueError("a part's cubes are not consecutive in Z-order")
            parts.append((depth, code, int(pos[0]), int(pos[-1])))
            return
        half = 1 << (root_bits - depth - 1)
        for ch in range(8):
            clo = lo + half * np.array([ch & 1, (ch >> 1) & 1, ch >> 2], np.int64)
            c = corner[members]
            inside = np.all((c >= clo) & (c < clo + half), axis=1)
            visit(depth + 1, code * 8 + ch, clo, members[inside])

    visit(0, 0, np.zeros(3, np.int64), np.arange(n))
    depth = np.array([p[0] for p in parts], np.int32)
    code = np.array([p[1] for p in parts], np.uint64)
    first = np.array([p[2] for p in parts], np.int64)
    last = np.array([p[3] for p in parts], np.int64)
    part = np.full(n, -1, np.int32)
    for j, (f, l) in enumerate(zip(first, last)):
        part[order[f:l + 1]] = j
    return depth, code, first, last, part
