"""Scene generators: cameras, depth maps, brick lists, chunk workloads.

Conventions shared with the C-ABI (``include/tgv.h``):

* Camera frame: ``Xc = R (X - C)``; pixel (i, j) covers ``[i, i+1) x [j, j+1)``.
  Pinhole (model 0): ``x = fx*Xc/Zc + cx``, ``y = fy*Yc/Zc + cy``; the rows of R
  are the camera's right, down and forward axes in world coordinates; depth
  maps store the camera-frame z-depth ``Zc`` of the observed surface point.
  Spherical (model 1, LIDAR scans): the rows of R are the scanner's x, y, z
  (z up); ``x = fx*azimuth + cx``, ``y = cy - fy*elevation``; maps store the
  range ``|Xc|`` of the observed point.
* Depth maps are float32, row-major, NaN where the ray hits nothing.
* A domain level is a list of 8^3 bricks given by integer brick coordinates;
  voxel (i, j, k) of brick (bx, by, bz) is the global voxel
  (8*bx+i, 8*by+j, 8*bz+k) whose centre is ``origin + (idx + 0.5) * h``.
* Seeds: configuration c gets seed 1000 + c (``CONFIG_SEEDS``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

CONFIG_SEEDS = {1: 1001, 2: 1002, 3: 1003, 4: 1004, 5: 1005}
BRICK = 8


# --------------------------------------------------------------------------- cameras
@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray  # (3, 3) float64, rows = right, down, forward (pinhole) / x, y, z (spherical)
    C: np.ndarray  # (3,) float64, camera centre
    width: int
    height: int
    model: int = 0  # 0 pinhole (z-depth maps), 1 spherical (LIDAR scan, range maps)

    def as_array(self) -> np.ndarray:
        """17 doubles: fx, fy, cx, cy, R (row-major), C, model."""
        return np.concatenate([[self.fx, self.fy, self.cx, self.cy],
                               np.asarray(self.R, np.float64).reshape(9),
                               np.asarray(self.C, np.float64).reshape(3), [float(self.model)]]).astype(np.float64)

    def ray_directions(self):
        """World direction per pixel centre.

        Pinhole: scaled so its camera-frame z is 1 (a point at parameter t along
        the ray has z-depth t).  Spherical: unit length (parameter t = range).
        Returns (H, W, 3) float64.
        """
        i = np.arange(self.width, dtype=np.float64) + 0.5
        j = np.arange(self.height, dtype=np.float64) + 0.5
        if self.model == 1:
            az, el = np.meshgrid((i - self.cx) / self.fx, (self.cy - j) / self.fy)
            dc = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=-1)
        else:
            xx, yy = np.meshgrid((i - self.cx) / self.fx, (j - self.cy) / self.fy)
            dc = np.stack([xx, yy, np.ones_like(xx)], axis=-1)
        return dc @ np.asarray(self.R, np.float64)  # (dc @ R) == (R^T dc^T)^T


def spherical_scanner(C, width: int, height: int, R=None) -> Camera:
    """A full 360 x 180 degree LIDAR scan as a spherical depth map of width x height
    pixels (equal angular steps), scanner axes R (default: the world axes)."""
    R = np.eye(3) if R is None else np.asarray(R, np.float64)
    return Camera(width / (2.0 * math.pi), height / math.pi, width / 2.0, height / 2.0, R,
                  np.asarray(C, np.float64), int(width), int(height), model=1)


def look_at(C, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    C = np.asarray(C, np.float64)
    f = np.asarray(target, np.float64) - C
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:  # looking along `up`: pick any orthogonal right axis
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    return np.stack([r, d, f])


def pinhole_intrinsics(width: int, height: int, hfov_deg: float):
    fx = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return fx, fx, width / 2.0, height / 2.0


# --------------------------------------------------------------------------- domains
@dataclass
class DomainDesc:
    """One level of a brick domain (active bricks plus optional frozen bricks)."""
    origin: np.ndarray
    h: float
    bricks: np.ndarray                     # (nb, 3) int32 brick coordinates
    frozen: Optional[np.ndarray] = None    # (nf, 3) int32
    frozen_u: Optional[np.ndarray] = None  # (nf, 512) float32
    frozen_v: Optional[np.ndarray] = None  # (nf, 3, 512) float32
    radius: float = 0.0                    # voxel radius for binning; <= 0 means h/2

    @property
    def nbricks(self) -> int:
        return int(self.bricks.shape[0])

    @property
    def nvox(self) -> int:
        return 512 * self.nbricks

    @property
    def nfrozen(self) -> int:
        return 0 if self.frozen is None else int(self.frozen.shape[0])


def dense_bricks(nbx: int, nby: int = None, nbz: int = None, offset=(0, 0, 0)) -> np.ndarray:
    """Brick coordinates of a dense box of bricks, x fastest."""
    nby = nbx if nby is None else nby
    nbz = nbx if nbz is None else nbz
    z, y, x = np.meshgrid(np.arange(nbz), np.arange(nby), np.arange(nbx), indexing="ij")
    c = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1) + np.asarray(offset)[None, :]
    return c.astype(np.int32)


@dataclass
class Scene:
    name: str
    domain: DomainDesc
    cameras: List[Camera]
    depths: List[np.ndarray]      # float32 (H, W), NaN = no sample
    nbins: int
    iterations: int
    alpha1: float = 1.0
    alpha0: float = 2.0
    votes: Sequence[int] = field(default_factory=list)
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------- depth maps
def plane_depth(width: int, height: int, depth: float) -> np.ndarray:
    """Fronto-parallel plane at camera z-depth `depth` (every pixel equal)."""
    return np.full((height, width), depth, dtype=np.float32)


def _sphere_hit(cam: Camera, centre, radius) -> np.ndarray:
    d = cam.ray_directions()
    oc = np.asarray(cam.C, np.float64) - np.asarray(centre, np.float64)
    a = np.einsum("hwk,hwk->hw", d, d)
    b = np.einsum("hwk,k->hw", d, oc)
    c = float(oc @ oc) - radius * radius
    disc = b * b - a * c
    t = np.full(a.shape, np.nan)
    ok = disc >= 0.0
    t[ok] = (-b[ok] - np.sqrt(disc[ok])) / a[ok]
    t[t <= 0.0] = np.nan
    return t


def sphere_scene(seed: int = CONFIG_SEEDS[1], n: int = 64, nmaps: int = 16, res: int = 128,
                 radius: float = 0.35, ring: float = 1.2, noise_frac: float = 0.005,
                 nbins: int = 8, iterations: int = 200) -> Scene:
    """Sphere of radius 0.35 centred in the unit cube, seen by a ring of pinhole cameras.

    Cameras: `nmaps` on a ring of radius `ring` about the centre, elevation
    alternating +20/-20 degrees, looking at the centre, 45 degree field of view.
    Depth: analytic ray/sphere z-depth plus N(0, (noise_frac*radius)^2).
    """
    rng = np.random.default_rng(seed)
    centre = np.array([0.5, 0.5, 0.5])
    fx, fy, cx, cy = pinhole_intrinsics(res, res, 45.0)
    cams, depths = [], []
    for k in range(nmaps):
        az = 2.0 * math.pi * k / nmaps
        el = math.radians(20.0 if k % 2 == 0 else -20.0)
        C = centre + ring * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cam = Camera(fx, fy, cx, cy, look_at(C, centre), C, res, res)
        t = _sphere_hit(cam, centre, radius)
        t = t + rng.normal(0.0, noise_frac * radius, size=t.shape)
        cams.append(cam)
        depths.append(t.astype(np.float32))
    nb = n // BRICK
    dom = DomainDesc(origin=np.zeros(3), h=1.0 / n, bricks=dense_bricks(nb))
    return Scene("sphere", dom, cams, depths, nbins, iterations, votes=[1] * nmaps,
                 meta=dict(centre=centre, radius=radius, seed=seed))


def lidar_sphere_scene(seed: int = CONFIG_SEEDS[1] + 100, n: int = 64, nscans: int = 4, width: int = 512,
                       height: int = 256, radius: float = 0.35, ring: float = 1.0, noise_frac: float = 0.001,
                       nbins: int = 8, iterations: int = 200) -> Scene:
    """The sphere of `sphere_scene` scanned by `nscans` spherical LIDAR scanners on a
    ring of radius `ring` about its centre (elevation alternating +10 / -10 degrees,
    scanner axes = world axes), full 360 x 180 degree range maps of width x height
    plus N(0, (noise_frac*radius)^2); vote 5 per scan (Sec. 3.4)."""
    rng = np.random.default_rng(seed)
    centre = np.array([0.5, 0.5, 0.5])
    cams, depths = [], []
    for k in range(nscans):
        az = 2.0 * math.pi * (k + 0.25) / nscans
        el = math.radians(10.0 if k % 2 == 0 else -10.0)
        C = centre + ring * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cam = spherical_scanner(C, width, height)
        t = _sphere_hit(cam, centre, radius)
        t = t + rng.normal(0.0, noise_frac * radius, size=t.shape)
        cams.append(cam)
        depths.append(t.astype(np.float32))
    nb = n // BRICK
    dom = DomainDesc(origin=np.zeros(3), h=1.0 / n, bricks=dense_bricks(nb))
    return Scene("lidar-sphere", dom, cams, depths, nbins, iterations, votes=[5] * nscans,
                 meta=dict(centre=centre, radius=radius, seed=seed))


# terrain --------------------------------------------------------------------------
@dataclass
class Terrain:
    amp: np.ndarray    # (6,)
    freq: np.ndarray   # (6, 2)
    phase: np.ndarray  # (6,)
    boxes: np.ndarray  # (nbox, 6): x0, x1, y0, y1, z0, z1
    base: float = 0.3

    def height(self, x, y, xp=np):
        z = self.base + 0.0 * x
        for k in range(self.amp.shape[0]):
            z = z + float(self.amp[k]) * xp.sin(2.0 * math.pi * (float(self.freq[k, 0]) * x + float(self.freq[k, 1]) * y)
                                                 + float(self.phase[k]))
        return z

    @property
    def lipschitz(self) -> float:
        return float(np.sum(2.0 * math.pi * np.linalg.norm(self.freq, axis=1) * self.amp))


def make_terrain(rng: np.random.Generator, nbox: int = 40) -> Terrain:
    amp = rng.uniform(0.01, 0.05, size=6)
    fmag = rng.uniform(1.0, 8.0, size=6)
    fdir = rng.uniform(0.0, 2.0 * math.pi, size=6)
    freq = np.stack([fmag * np.cos(fdir), fmag * np.sin(fdir)], axis=1)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=6)
    t = Terrain(amp, freq, phase, np.zeros((0, 6)))
    boxes = []
    for _ in range(nbox):
        sx, sy = rng.uniform(0.02, 0.12, size=2)
        cxb, cyb = rng.uniform(0.1, 0.9, size=2)
        top = float(t.height(np.array(cxb), np.array(cyb))) + rng.uniform(0.05, 0.3)
        boxes.append([cxb - sx / 2, cxb + sx / 2, cyb - sy / 2, cyb + sy / 2, -1.0, top])
    t.boxes = np.array(boxes, dtype=np.float64)
    return t


def _torch():
    import torch
    return torch


def _terrain_depth_torch(terrain: Terrain, cams: List[Camera], step: float, device) -> List[np.ndarray]:
    """Ray-cast the height field (Lipschitz-bounded march + bisection) and the boxes.

    All rays of all cameras are marched together; returns one (H, W) float64 z-depth
    map per camera (NaN where the ray leaves the scene without a hit).
    """
    torch = _torch()
    d = torch.cat([torch.as_tensor(c.ray_directions().reshape(-1, 3), dtype=torch.float64) for c in cams]).to(device)
    C = torch.cat([torch.as_tensor(np.asarray(c.C, np.float64)[None, :].repeat(c.width * c.height, 0))
                   for c in cams]).to(device)
    n = d.shape[0]
    ztop = terrain.base + float(np.sum(terrain.amp)) + 1e-6
    zbot = terrain.base - float(np.sum(terrain.amp)) - 1e-6
    L = terrain.lipschitz
    dz = d[:, 2]
    dxy = torch.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    dn = torch.sqrt(dz * dz + dxy * dxy)
    down = dz < -1e-9
    big = torch.full((n,), float("inf"), dtype=torch.float64, device=device)
    safe_dz = torch.where(down, dz, -torch.ones_like(dz))
    t0 = torch.where(down, torch.clamp((ztop - C[:, 2]) / safe_dz, min=0.0), big)
    t1 = torch.where(down, (zbot - C[:, 2]) / safe_dz, big)

    def g(t, idx):
        p = C[idx] + t[:, None] * d[idx]
        return p[:, 2] - terrain.height(p[:, 0], p[:, 1], xp=torch)

    t_hit = big.clone()
    idx = torch.nonzero(down).squeeze(1)
    t = t0[idx].clone()
    gv = g(t, idx)
    denom = (-dz[idx]) + L * dxy[idx]
    dtmin = step / dn[idx]
    for _ in range(200000):
        if idx.numel() == 0:
            break
        tn = t + torch.maximum(gv / denom, dtmin)
        gn = g(tn, idx)
        crossed = gn <= 0.0
        if bool(crossed.any()):
            lo, hi = t[crossed], tn[crossed]
            ci = idx[crossed]
            for _b in range(40):
                mid = 0.5 * (lo + hi)
                below = g(mid, ci) <= 0.0
                hi = torch.where(below, mid, hi)
                lo = torch.where(below, lo, mid)
            t_hit[ci] = hi
        keep = (~crossed) & (tn <= t1[idx])
        idx, t, gv = idx[keep], tn[keep], gn[keep]
        denom, dtmin = denom[keep], dtmin[keep]
    # boxes: slab test
    if terrain.boxes.shape[0]:
        inv = 1.0 / torch.where(d.abs() < 1e-300, torch.full_like(d, 1e-300), d)
        for bx in terrain.boxes:
            lo = torch.as_tensor(bx[[0, 2, 4]], dtype=torch.float64, device=device)
            hi = torch.as_tensor(bx[[1, 3, 5]], dtype=torch.float64, device=device)
            ta = (lo[None, :] - C) * inv
            tb = (hi[None, :] - C) * inv
            tnear = torch.minimum(ta, tb).max(dim=1).values
            tfar = torch.maximum(ta, tb).min(dim=1).values
            hit = (tnear <= tfar) & (tnear > 0.0)
            t_hit = torch.where(hit & (tnear < t_hit), tnear, t_hit)
    t_hit = torch.where(torch.isinf(t_hit), torch.full_like(t_hit, float("nan")), t_hit).cpu().numpy()
    out, o = [], 0
    for c in cams:
        out.append(t_hit[o:o + c.width * c.height].reshape(c.height, c.width))
        o += c.width * c.height
    return out


def terrain_scene(seed: int = CONFIG_SEEDS[2], n: int = 256, nmaps: int = 64, res: int = 512,
                  nbins: int = 10, iterations: int = 500, noise_vox: float = 0.3,
                  outlier_frac: float = 0.05, device=None) -> Scene:
    """Terrain of 6 random sinusoids plus 40 box buildings over the unit square.

    Cameras: 16 nadir cameras on a 4x4 grid at altitude 1.5 (40 degree field of
    view) and 48 oblique cameras (4 azimuths x 12, tilted 40 degrees from nadir,
    50 degree field of view).  If `nmaps` < 64 the first `nmaps` of the interleaved
    list are used.  Depth noise N(0, (noise_vox*h)^2); a fraction `outlier_frac`
    of valid pixels is replaced by U(min, max) of that map's depths.
    """
    torch = _torch()
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    rng = np.random.default_rng(seed)
    terrain = make_terrain(rng)
    h = 1.0 / n
    cams: List[Camera] = []
    fxn = pinhole_intrinsics(res, res, 40.0)
    for gy in range(4):
        for gx in range(4):
            C = np.array([0.125 + 0.25 * gx, 0.125 + 0.25 * gy, 1.5])
            cams.append(Camera(*fxn, look_at(C, C - np.array([0, 0, 1.0]), up=(0, 1, 0)), C, res, res))
    fxo = pinhole_intrinsics(res, res, 50.0)
    tilt = math.radians(40.0)
    obl = []
    for k in range(4):
        az = k * math.pi / 2
        for gy in range(3):
            for gx in range(4):
                tx, ty = 0.2 + 0.2 * gx - 0.5, 0.25 + 0.25 * gy - 0.5
                ca, sa = math.cos(az), math.sin(az)
                T = np.array([0.5 + ca * tx - sa * ty, 0.5 + sa * tx + ca * ty, terrain.base])
                off = 1.2 * math.tan(tilt)
                C = T + np.array([-ca * off, -sa * off, 1.2])
                obl.append(Camera(*fxo, look_at(C, T), C, res, res))
    # interleave so that a prefix of the list mixes nadir and oblique views
    allc = []
    for k in range(48):
        if k % 3 == 0 and k // 3 < 16:
            allc.append(cams[k // 3])
        allc.append(obl[k])
    cams = allc[:nmaps]
    depths = []
    for t in _terrain_depth_torch(terrain, cams, step=h / 4, device=device):
        valid = np.isfinite(t)
        t = t + rng.normal(0.0, noise_vox * h, size=t.shape)
        if valid.any():
            lo, hi = float(np.nanmin(t[valid])), float(np.nanmax(t[valid]))
            out = (rng.random(t.shape) < outlier_frac) & valid
            t[out] = rng.uniform(lo, hi, size=int(out.sum()))
        depths.append(t.astype(np.float32))
    dom = DomainDesc(origin=np.zeros(3), h=h, bricks=dense_bricks(n // BRICK))
    return Scene("terrain", dom, cams, depths, nbins, iterations, votes=[1] * len(cams),
                 meta=dict(seed=seed, terrain=terrain))


def terrain_lidar_scans(terrain: "Terrain", nscans: int = 16, width: int = 2048, height: int = 1024,
                        h: float = 1.0 / 256, mast: float = 0.02, noise_vox: float = 0.1, seed: int = 1102,
                        device=None):
    """Ground LIDAR scans of a terrain (the terrestrial scans of the paper's mixed
    datasets): `nscans` scanners on a square grid over the central 0.8 x 0.8 of the
    unit square, `mast` above the ground (moved off any building footprint), full
    360 x 180 degree range maps of width x height, noise N(0, (noise_vox*h)^2).
    Returns (cameras, range maps)."""
    torch = _torch()
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    rng = np.random.default_rng(seed)
    g = int(round(math.sqrt(nscans)))
    cams = []
    for k in range(nscans):
        x, y = 0.1 + 0.8 * ((k % g) + 0.5) / g, 0.1 + 0.8 * ((k // g) + 0.5) / g
        for _ in range(64):  # step off building footprints
            inside = [(b[0] <= x <= b[1] and b[2] <= y <= b[3]) for b in terrain.boxes]
            if not any(inside):
                break
            x, y = x + 0.013, y + 0.007
        z = float(terrain.height(np.array([x]), np.array([y]))[0]) + mast
        cams.append(spherical_scanner(np.array([x, y, z]), width, height))
    depths = []
    for t in _terrain_depth_torch(terrain, cams, step=h / 4, device=device):
        t = t + rng.normal(0.0, noise_vox * h, size=t.shape)
        depths.append(t.astype(np.float32))
    return cams, depths


# --------------------------------------------------------------------------- histograms
def random_histograms(rng: np.random.Generator, nvox: int, nbins: int, max_count: int = 20,
                      empty_frac: float = 0.1) -> np.ndarray:
    """Uniform random per-voxel counts (uint32, (nvox, nbins)); a fraction of voxels empty."""
    hst = rng.integers(0, max_count + 1, size=(nvox, nbins)).astype(np.uint32)
    hst[rng.random(nvox) < empty_frac] = 0
    return hst


# --------------------------------------------------------------------------- chunk workloads
@dataclass
class ChunkSpec:
    """One chunk-solve request: a box of bricks with a frozen one-brick face shell."""
    domain: DomainDesc
    hist: object       # (nvox, nbins) counts: uint32 numpy, int32 torch, or None
    nbins: int
    iterations: int
    arrival: float = 0.0
    meta: dict = field(default_factory=dict)


def _box_dims(nb: int, rng) -> tuple:
    s = max(1, round(nb ** (1.0 / 3.0)))
    a, b = s, s
    c = max(1, round(nb / (a * b)))
    return a, b, c


def _synthetic_votes(s_vox: np.ndarray, nbins: int, rng, views: int) -> np.ndarray:
    """Synthetic per-voxel counts from the height above a surface (voxel units).

    Statistical input model (not Alg. 1): each of `views` virtual observations
    of a voxel with height s above the surface lands in a bin drawn around
    (n-1)/2 + s*(n-1)/6 with unit Gaussian jitter, clipped to the bin range;
    voxels deeper than 9 voxels below the surface get no observations; 5% of
    observations are uniform outliers.
    """
    nv = s_vox.shape[0]
    flat = np.zeros(nv * nbins, np.int64)
    seen = s_vox > -9.0
    centre = (nbins - 1) / 2.0 + s_vox * (nbins - 1) / 6.0
    base = np.arange(nv, dtype=np.int64) * nbins
    for _ in range(views):
        b = np.rint(centre + rng.normal(0.0, 1.0, size=nv))
        outl = rng.random(nv) < 0.05
        b[outl] = rng.integers(0, nbins, size=int(outl.sum()))
        b = np.clip(b, 0, nbins - 1).astype(np.int64)
        flat += np.bincount((base + b)[seen], minlength=nv * nbins)
    return flat.reshape(nv, nbins).astype(np.uint32)


def synthetic_votes_torch(s_vox, nbins: int, seed: int, views: int = 12):
    """Same statistical vote model as _synthetic_votes, drawn with torch on s_vox's device.

    Returns int32 counts (nvox, nbins) on that device.
    """
    torch = _torch()
    dev = s_vox.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    nv = s_vox.shape[0]
    out = torch.zeros(nv * nbins, dtype=torch.int32, device=dev)
    seen = s_vox > -9.0
    centre = (nbins - 1) / 2.0 + s_vox * ((nbins - 1) / 6.0)
    base = torch.arange(nv, device=dev, dtype=torch.int64) * nbins
    ones = seen.to(torch.int32)
    for _ in range(views):
        b = torch.round(centre + torch.randn(nv, generator=gen, device=dev, dtype=centre.dtype))
        outl = torch.rand(nv, generator=gen, device=dev) < 0.05
        b = torch.where(outl, torch.randint(0, nbins, (nv,), generator=gen, device=dev).to(b.dtype), b)
        b = b.clamp(0, nbins - 1).to(torch.int64)
        out.index_add_(0, base + b, ones)
    return out.view(nv, nbins)


def chunk_heights(terrain: "Terrain", bricks: np.ndarray, h: float, device=None):
    """Height above the terrain surface, in voxels, of every voxel of `bricks` (brick order)."""
    if device is None:
        li = np.arange(512)
        lx, ly, lz = li % 8, (li // 8) % 8, li // 64
        gx = (bricks[:, 0:1] * 8 + lx[None, :] + 0.5) * h
        gy = (bricks[:, 1:2] * 8 + ly[None, :] + 0.5) * h
        gz = (bricks[:, 2:3] * 8 + lz[None, :] + 0.5) * h
        return ((gz - terrain.height(gx, gy)) / h).reshape(-1)
    torch = _torch()
    bt = torch.as_tensor(bricks, dtype=torch.float64, device=device)
    li = torch.arange(512, device=device)
    lx, ly, lz = (li % 8).double(), ((li // 8) % 8).double(), (li // 64).double()
    gx = (bt[:, 0:1] * 8 + lx[None, :] + 0.5) * h
    gy = (bt[:, 1:2] * 8 + ly[None, :] + 0.5) * h
    gz = (bt[:, 2:3] * 8 + lz[None, :] + 0.5) * h
    return ((gz - terrain.height(gx, gy, xp=torch)) / h).reshape(-1)


def chunk_workload(seed: int, nchunks: int, min_vox: int, max_vox: int, nbins_range=(10, 10),
                   iters_range=(300, 300), rate: float = 0.0, max_total_vox: Optional[int] = None,
                   views: int = 12, hist: str = "numpy", device=None) -> List[ChunkSpec]:
    """Chunks cut from an unbounded terrain-style scene (sum of 6 sinusoids).

    Active voxel count log-uniform in [min_vox, max_vox], rounded to whole
    bricks and shaped as a near-cubic box of bricks placed at a random position;
    its frozen halo is every brick face-adjacent to the box, carrying
    u = clip(s/3, -1, 1) (s = height above the surface in voxels) and v = 0.
    `rate` > 0 draws Poisson arrival times (requests/s).
    hist: "numpy" (host counts now), "torch" (int32 counts on `device` now) or
    "none" (hist = None; draw later with chunk_histogram(spec)).
    """
    rng = np.random.default_rng(seed)
    terrain = make_terrain(rng, nbox=0)
    specs = []
    t_arr = 0.0
    for c in range(nchunks):
        nvox = math.exp(rng.uniform(math.log(min_vox), math.log(max_vox)))
        nb = max(1, int(round(nvox / 512)))
        a, b, cdim = _box_dims(nb, rng)
        n = 256
        h = 1.0 / n
        off = np.array([rng.integers(0, 32), rng.integers(0, 32), 0])
        bricks = dense_bricks(a, b, cdim, offset=off)
        # vertical placement: centre the box on the terrain height at its centre
        cxw = (off[0] + a / 2) * 8 * h
        cyw = (off[1] + b / 2) * 8 * h
        zc = float(terrain.height(np.array(cxw), np.array(cyw)))
        oz = int(round(zc / (8 * h) - cdim / 2))
        bricks[:, 2] += oz
        # frozen face shell
        act = {tuple(x) for x in bricks.tolist()}
        fro = set()
        for x in act:
            for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                y = (x[0] + dx, x[1] + dy, x[2] + dz)
                if y not in act:
                    fro.add(y)
        frozen = np.array(sorted(fro), dtype=np.int32).reshape(-1, 3)
        nbins = int(rng.integers(nbins_range[0], nbins_range[1] + 1))
        iters = int(rng.integers(iters_range[0], iters_range[1] + 1))

        def heights(bc):
            li = np.arange(512)
            lx, ly, lz = li % 8, (li // 8) % 8, li // 64
            gx = (bc[:, 0:1] * 8 + lx[None, :] + 0.5) * h
            gy = (bc[:, 1:2] * 8 + ly[None, :] + 0.5) * h
            gz = (bc[:, 2:3] * 8 + lz[None, :] + 0.5) * h
            return (gz - terrain.height(gx, gy)) / h  # (nb, 512) voxel units

        vote_seed = int(rng.integers(0, 2**31 - 1))
        if hist == "numpy":
            hst = _synthetic_votes(heights(bricks).reshape(-1), nbins, np.random.default_rng(vote_seed), views)
        elif hist == "torch":
            hst = synthetic_votes_torch(chunk_heights(terrain, bricks, h, device), nbins, vote_seed, views)
        else:
            hst = None
        fu = np.clip(heights(frozen) / 3.0, -1.0, 1.0).astype(np.float32) if len(frozen) else None
        fv = np.zeros((len(frozen), 3, 512), np.float32) if len(frozen) else None
        dom = DomainDesc(origin=np.zeros(3), h=h, bricks=bricks,
                         frozen=frozen if len(frozen) else None, frozen_u=fu, frozen_v=fv)
        if rate > 0:
            t_arr += rng.exponential(1.0 / rate)
        sp = ChunkSpec(dom, hst, nbins, iters, t_arr)
        sp.meta = dict(terrain=terrain, vote_seed=vote_seed, views=views)
        specs.append(sp)
    return specs


def chunk_histogram(spec: "ChunkSpec", device):
    """Draws the counts of a chunk made with hist="none" (int32 (nvox, nbins) on `device`)."""
    m = spec.meta
    return synthetic_votes_torch(chunk_heights(m["terrain"], spec.domain.bricks, spec.domain.h, device), spec.nbins,
                                 m["vote_seed"], m["views"])


# --------------------------------------------------------------------------- multi-level scene
@dataclass
class Blob:
    """Union of ellipsoids (centre, rotation, semi-axes) and tori (centre, axis, R, r)."""
    ell_c: np.ndarray  # (ne, 3)
    ell_q: np.ndarray  # (ne, 3, 3) columns = local axes
    ell_a: np.ndarray  # (ne, 3)
    tor_c: np.ndarray  # (nt, 3)
    tor_n: np.ndarray  # (nt, 3)
    tor_R: np.ndarray  # (nt,)
    tor_r: np.ndarray  # (nt,)

    @property
    def bound(self):
        lo = np.minimum((self.ell_c - self.ell_a.max(1, keepdims=True)).min(0),
                        (self.tor_c - (self.tor_R + self.tor_r)[:, None]).min(0))
        hi = np.maximum((self.ell_c + self.ell_a.max(1, keepdims=True)).max(0),
                        (self.tor_c + (self.tor_R + self.tor_r)[:, None]).max(0))
        return lo, hi

    def sdf(self, p, xp=np):
        """Approximate signed distance (exact for the tori, the usual scaled-sphere bound for ellipsoids)."""
        d = None
        for k in range(self.ell_c.shape[0]):
            q = (p - self.ell_c[k]) @ self.ell_q[k] if xp is np else (p - xp.as_tensor(self.ell_c[k], device=p.device)) @ xp.as_tensor(self.ell_q[k], device=p.device)
            a = self.ell_a[k]
            a_t = a if xp is np else xp.as_tensor(a, device=p.device)
            k0 = (((q / a_t) ** 2).sum(-1)) ** 0.5
            k1 = (((q / a_t ** 2) ** 2).sum(-1)) ** 0.5
            e = k0 * (k0 - 1.0) / (k1 + 1e-12)
            d = e if d is None else (xp.minimum(d, e))
        for k in range(self.tor_c.shape[0]):
            c = self.tor_c[k] if xp is np else xp.as_tensor(self.tor_c[k], device=p.device)
            n = self.tor_n[k] if xp is np else xp.as_tensor(self.tor_n[k], device=p.device)
            x = p - c
            h = (x * n).sum(-1)
            perp = ((x * x).sum(-1) - h * h).clip(0) ** 0.5 if xp is np else (((x * x).sum(-1) - h * h).clamp(min=0)) ** 0.5
            e = ((perp - self.tor_R[k]) ** 2 + h * h) ** 0.5 - self.tor_r[k]
            d = xp.minimum(d, e)
        return d


def make_blob(rng: np.random.Generator, centre: np.ndarray, radius: float) -> Blob:
    def rot():
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        return q
    ne, nt = 5, 3
    ell_c = centre + rng.uniform(-0.35, 0.35, size=(ne, 3)) * radius
    ell_q = np.stack([rot() for _ in range(ne)])
    ell_a = rng.uniform(0.25, 0.6, size=(ne, 3)) * radius
    tor_c = centre + rng.uniform(-0.3, 0.3, size=(nt, 3)) * radius
    tor_n = rng.normal(size=(nt, 3))
    tor_n /= np.linalg.norm(tor_n, axis=1, keepdims=True)
    tor_R = rng.uniform(0.3, 0.5, size=nt) * radius
    tor_r = rng.uniform(0.06, 0.12, size=nt) * radius
    return Blob(ell_c, ell_q, ell_a, tor_c, tor_n, tor_R, tor_r)


def _blob_hits_torch(blob: Blob, C, d, step_floor: float, device):
    """First hit parameter of rays C + t d with the blob (inf where none)."""
    torch = _torch()
    n = d.shape[0]
    inf = torch.full((n,), float("inf"), dtype=torch.float64, device=device)
    t_best = inf.clone()
    for k in range(blob.ell_c.shape[0]):  # ellipsoids: unit-sphere intersection in local frame
        Q = torch.as_tensor(blob.ell_q[k], dtype=torch.float64, device=device)
        a = torch.as_tensor(blob.ell_a[k], dtype=torch.float64, device=device)
        c = torch.as_tensor(blob.ell_c[k], dtype=torch.float64, device=device)
        o2 = ((C - c) @ Q) / a
        d2 = (d @ Q) / a
        A = (d2 * d2).sum(-1)
        B = (o2 * d2).sum(-1)
        Cc = (o2 * o2).sum(-1) - 1.0
        disc = B * B - A * Cc
        ok = disc >= 0
        t = (-B - torch.sqrt(disc.clamp(min=0))) / A
        t = torch.where(ok & (t > 0), t, inf)
        t_best = torch.minimum(t_best, t)
    # tori: sphere tracing of the exact distance, started at the bounding sphere
    for k in range(blob.tor_c.shape[0]):
        c = torch.as_tensor(blob.tor_c[k], dtype=torch.float64, device=device)
        nrm = torch.as_tensor(blob.tor_n[k], dtype=torch.float64, device=device)
        R, r = float(blob.tor_R[k]), float(blob.tor_r[k])
        dn = torch.sqrt((d * d).sum(-1))
        oc = C - c
        bb = (oc * d).sum(-1) / dn
        cc = (oc * oc).sum(-1) - (R + r) ** 2
        disc = bb * bb - cc
        t = torch.where(disc > 0, (-bb - torch.sqrt(disc.clamp(min=0))).clamp(min=0) / dn, inf)
        idx = torch.nonzero(torch.isfinite(t)).squeeze(1)
        tt = t[idx]
        hit = torch.zeros(idx.shape[0], dtype=torch.bool, device=device)
        for _ in range(200):
            p = C[idx] + tt[:, None] * d[idx]
            x = p - c
            h = (x * nrm).sum(-1)
            perp = torch.sqrt(((x * x).sum(-1) - h * h).clamp(min=0))
            sd = torch.sqrt((perp - R) ** 2 + h * h) - r
            hit = hit | (sd < 1e-7)
            tt = torch.where(hit, tt, tt + sd / dn[idx])
            if bool(hit.all()):
                break
        far = (~hit) | (tt > t_best[idx])
        t_best[idx] = torch.where(far, t_best[idx], tt)
    return t_best


def multilevel_scene(seed: int = CONFIG_SEEDS[3], n0: int = 1024, blob_radius_vox: float = 56.0,
                     nmaps_aerial: int = 192, nmaps_ring: int = 64, res: int = 1024, nbins: int = 10,
                     iterations: int = 200, noise_vox: float = 0.3, footprint: float = 0.75, device=None) -> dict:
    """Sparse three-level brick domain: terrain at level 0 (voxel h0 = 1/n0 over the unit
    square), a statue-like blob (5 ellipsoids + 3 tori, radius `blob_radius_vox` level-0
    voxels) floating above it refined to level 2 (h0/4), and a level-1 (h0/2) transition
    shell around the blob.  Active bricks of a level: brick centres within the band
    |signed distance| <= eta + brick half-diagonal (+ a 2-brick dilation on level 1); the
    frozen shell of levels 1 and 2: bricks face-adjacent to the level's active bricks.
    Level 0 covers the central `footprint` x `footprint` part of the unit square.
    Maps: `nmaps_aerial` over the terrain (nadir and oblique) and `nmaps_ring` on two rings
    around the blob, all res x res; z-depth noise N(0, (noise_vox * h_level)^2) with h of the
    finest level the map sees.
    """
    torch = _torch()
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    rng = np.random.default_rng(seed)
    terrain = make_terrain(rng, nbox=0)
    h0 = 1.0 / n0
    hs = [h0, h0 / 2, h0 / 4]
    top = terrain.base + float(np.sum(terrain.amp))
    bc = np.array([0.5, 0.5, top + 1.6 * blob_radius_vox * h0])
    blob = make_blob(rng, bc, blob_radius_vox * h0)
    blo, bhi = blob.bound

    def brick_centres(bricks, h):
        return (bricks.astype(np.float64) * 8 + 4.0) * h

    def terrain_sd(p):
        """Vertical offset over the local slope: (z - H) / sqrt(1 + |grad H|^2)."""
        gz = terrain.height(p[:, 0], p[:, 1])
        e = 1e-5
        gx = (terrain.height(p[:, 0] + e, p[:, 1]) - terrain.height(p[:, 0] - e, p[:, 1])) / (2 * e)
        gy = (terrain.height(p[:, 0], p[:, 1] + e) - terrain.height(p[:, 0], p[:, 1] - e)) / (2 * e)
        return (p[:, 2] - gz) / np.sqrt(1.0 + gx * gx + gy * gy)

    # level 0: terrain band over the unit square, plus the blob band at the coarse level
    nb0 = n0 // 8
    f0 = int(round(nb0 * (1.0 - footprint) / 2.0))
    nbf = nb0 - 2 * f0
    band0 = (9.0 + 4.0 * np.sqrt(3.0)) * h0
    zlo = int(np.floor((terrain.base - float(np.sum(terrain.amp)) - band0) / (8 * h0))) - 1
    zhi = int(np.ceil((bhi[2] + band0) / (8 * h0))) + 1
    cand = dense_bricks(nbf, nbf, zhi - zlo, offset=(f0, f0, zlo))
    cc = brick_centres(cand, h0)
    sd = np.minimum(np.abs(terrain_sd(cc)), np.abs(blob.sdf(cc)))
    lv0 = cand[sd <= band0]
    levels = [lv0]
    # levels 1 and 2: bricks in the blob's bounding box (dilated) near the blob surface
    for l, dil in ((1, 2), (2, 0)):
        h = hs[l]
        band = (9.0 + 4.0 * np.sqrt(3.0)) * h + dil * 8 * h
        lo = np.floor((blo - band) / (8 * h)).astype(int) - 1
        hi = np.ceil((bhi + band) / (8 * h)).astype(int) + 1
        cand = dense_bricks(*(hi - lo), offset=tuple(lo))
        cc = brick_centres(cand, h)
        levels.append(cand[np.abs(blob.sdf(cc)) <= band])
    descs = []
    for l, act in enumerate(levels):
        frozen = None
        if l > 0:
            s = {tuple(x) for x in act.tolist()}
            fro = set()
            for x in s:
                for dd in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    y = (x[0] + dd[0], x[1] + dd[1], x[2] + dd[2])
                    if y not in s:
                        fro.add(y)
            frozen = np.array(sorted(fro), np.int32).reshape(-1, 3)
        descs.append(DomainDesc(np.zeros(3), hs[l], act.astype(np.int32), frozen=frozen))
    # cameras
    cams: List[Camera] = []
    fxa = pinhole_intrinsics(res, res, 40.0)
    na = nmaps_aerial
    side = int(np.ceil(np.sqrt(max(1, na // 3))))
    for k in range(na):
        if k % 3 == 0:  # nadir on a grid
            g = k // 3
            gx, gy = g % side, (g // side) % side
            C = np.array([(gx + 0.5) / side, (gy + 0.5) / side, 1.5])
            cams.append(Camera(*fxa, look_at(C, C - np.array([0, 0, 1.0]), up=(0, 1, 0)), C, res, res))
        else:  # oblique, 40 degrees, azimuth cycling
            az = 2 * np.pi * rng.random()
            T = np.array([rng.uniform(0.1, 0.9), rng.uniform(0.1, 0.9), terrain.base])
            off = 1.2 * np.tan(np.radians(40.0))
            C = T + np.array([-np.cos(az) * off, -np.sin(az) * off, 1.2])
            cams.append(Camera(*fxa, look_at(C, T), C, res, res))
    fxr = pinhole_intrinsics(res, res, 35.0)
    rb = float(np.max(bhi - blo))
    for k in range(nmaps_ring):
        az = 2 * np.pi * k / max(1, nmaps_ring // 2)
        el = np.radians(25.0 if k % 2 == 0 else 55.0)
        dist = 2.2 * rb
        C = bc + dist * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        cams.append(Camera(*fxr, look_at(C, bc), C, res, res))
    # ray casting: terrain and blob, nearest hit
    depths = []
    for k0 in range(0, len(cams), 16):
        batch = cams[k0:k0 + 16]
        t_ter = _terrain_depth_torch(terrain, batch, step=hs[0], device=device)
        d = torch.cat([torch.as_tensor(c.ray_directions().reshape(-1, 3), dtype=torch.float64) for c in batch]).to(device)
        C = torch.cat([torch.as_tensor(np.asarray(c.C, np.float64)[None, :].repeat(c.width * c.height, 0))
                       for c in batch]).to(device)
        t_blob = _blob_hits_torch(blob, C, d, hs[2], device).cpu().numpy()
        o = 0
        for c, tt in zip(batch, t_ter):
            tb = t_blob[o:o + c.width * c.height].reshape(c.height, c.width)
            o += c.width * c.height
            t = np.where(np.isnan(tt), tb, np.minimum(np.nan_to_num(tt, nan=np.inf), tb))
            t = np.where(np.isfinite(t), t, np.nan)
            valid = np.isfinite(t)
            t = t + rng.normal(0.0, noise_vox * hs[2], size=t.shape)
            t[~valid] = np.nan
            depths.append(t.astype(np.float32))
    return dict(levels=descs, cameras=cams, depths=depths, nbins=nbins, iterations=iterations,
                terrain=terrain, blob=blob, h=hs, seed=seed)
