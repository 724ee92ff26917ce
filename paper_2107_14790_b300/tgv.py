"""ctypes binding of the C-ABI in include/tgv.h (argument marshalling only).

Every function named ``tgv_*`` here calls the C entry point of the same name;
all arithmetic runs in the library's CUDA kernels.  The library must have been
built (``python -m paper_2107_14790_b300.build``); there is no fallback: a
missing or unloadable ``libtgv.so`` raises ImportError.

Device buffers are passed as raw pointers (``torch.Tensor.data_ptr()``); host
buffers as numpy arrays.  PyTorch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtgv.so")

TGV_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "budget exceeded", 4: "CUDA error",
          5: "device wait timed out", 6: "domain in error state", 7: "unsupported"}
STORAGE = {"fp32": 0, "bf16": 1, "fp16": 2, "fx16": 3}
HIST_FORMS = {"gather": 0, "scatter": 1}
FIELDS = {"u": (0, 1), "ubar": (1, 1), "v": (2, 3), "vbar": (3, 3), "p": (4, 3), "q": (5, 6)}


class TgvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class tgv_params(ctypes.Structure):
    _fields_ = [("nbins", ctypes.c_int32), ("alpha1", ctypes.c_float), ("alpha0", ctypes.c_float),
                ("lam", ctypes.c_float), ("tau", ctypes.c_float), ("sigma", ctypes.c_float),
                ("storage", ctypes.c_int32), ("clamp_u", ctypes.c_int32), ("centres", ctypes.c_int32),
                ("box_v", ctypes.c_float), ("iter_kernel", ctypes.c_int32),
                ("x_run", ctypes.c_int32), ("hist_form", ctypes.c_int32), ("wait_cycles", ctypes.c_int64),
                ("wait_test", ctypes.c_int32)]


class tgv_level_desc(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("h", ctypes.c_double), ("radius", ctypes.c_double),
                ("nbricks", ctypes.c_int64), ("brick_coords", ctypes.c_void_p),
                ("nfrozen", ctypes.c_int64), ("frozen_coords", ctypes.c_void_p),
                ("frozen_u", ctypes.c_void_p), ("frozen_v", ctypes.c_void_p)]


class tgv_camera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("R", ctypes.c_double * 9), ("C", ctypes.c_double * 3), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("model", ctypes.c_int32)]


class tgv_state_view(ctypes.Structure):
    _fields_ = [("nbricks", ctypes.c_int64), ("nall", ctypes.c_int64), ("u", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("p", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("hist", ctypes.c_void_p), ("nbr", ctypes.c_void_p)]


class tgv_server_cfg(ctypes.Structure):
    _fields_ = [("capacity_bricks", ctypes.c_int64), ("capacity_frozen", ctypes.c_int64),
                ("staging_bytes", ctypes.c_int64)]


_lib = None


def lib() -> ctypes.CDLL:
    """Loads libtgv.so once; raises ImportError if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} not built: run `python -m paper_2107_14790_b300.build`")
    L = ctypes.CDLL(_LIB_PATH)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "tgv_default_params": (i32, [P]),
        "tgv_create_domain": (i32, [P, i32, P, P, P]),
        "tgv_destroy_domain": (None, [P]),
        "tgv_accumulate_depthmap": (i32, [P, i32, P, P, i64, u32]),
        "tgv_accumulate_depthmaps": (i32, [P, i32, P, i32, P, i64, i64, P]),
        "tgv_solve": (i32, [P, i32, i32, P]),
        "tgv_energy": (i32, [P, i32, P]),
        "tgv_extract_field": (i32, [P, i32, i32, P, i64]),
        "tgv_set_field": (i32, [P, i32, i32, P, i64]),
        "tgv_extract_histograms": (i32, [P, i32, P, i64]),
        "tgv_set_histograms": (i32, [P, i32, P, i64]),
        "tgv_reset": (i32, [P, i32, i32]),
        "tgv_prolong": (i32, [P, i32]),
        "tgv_synchronize": (i32, [P]),
        "tgv_domain_bytes": (i64, [P]),
        "tgv_level_voxels": (i64, [P, i32]),
        "tgv_launch_count": (i64, [P]),
        "tgv_pair_run_length": (i32, [P, i64, P, i64, i64, i32, P]),
        "tgv_extract_mesh": (i32, [P, i32, P, P]),
        "tgv_octree_build": (i32, [P, P, i32, P, i64, i64, P, P]),
        "tgv_composite_create": (i32, [P, P]),
        "tgv_composite_solve": (i32, [P, i32]),
        "tgv_composite_leaves": (i64, [P]),
        "tgv_composite_level_leaves": (i64, [P, i32]),
        "tgv_composite_extract": (i32, [P, P, i64]),
        "tgv_composite_scatter": (i32, [P]),
        "tgv_composite_launch_count": (i64, [P]),
        "tgv_composite_treetop": (i32, [P, i32, i64, P]),
        "tgv_composite_treetop_parts": (i32, [P, P, P, P, P, P]),
        "tgv_composite_destroy": (None, [P]),
        "tgv_octree_levels": (i32, [P]),
        "tgv_octree_samples": (i64, [P]),
        "tgv_octree_level": (i32, [P, i32, P, P, P, P]),
        "tgv_octree_bricks": (i32, [P, i32, P, P]),
        "tgv_octree_destroy": (None, [P]),
        "tgv_copy_mesh": (i32, [P, P, i64, P, i64]),
        "tgv_energy_noalloc": (i32, [P, P, P, P]),
        "tgv_solve_graph": (i32, [P, i32, i32, P]),
        "tgv_solve_chunks": (i32, [P, i32, i32, P, P, i32]),
        "tgv_set_work_list": (i32, [P, i32, P, i64]),
        "tgv_server_create": (i32, [P, P, P, P]),
        "tgv_server_submit": (i32, [P, P, P, i32, P]),
        "tgv_server_step": (i32, [P, i32, P]),
        "tgv_server_poll": (i32, [P, ctypes.c_uint64, P]),
        "tgv_server_extract": (i32, [P, ctypes.c_uint64, P, i64]),
        "tgv_server_free_bricks": (i64, [P]),
        "tgv_server_running": (i64, [P]),
        "tgv_server_voxel_updates": (i64, [P]),
        "tgv_server_synchronize": (i32, [P]),
        "tgv_server_last_error": (ctypes.c_char_p, [P]),
        "tgv_server_destroy": (None, [P]),
        "tgv_status_string": (ctypes.c_char_p, [i32]),
        "tgv_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols() -> Sequence[str]:
    """Names of the C entry points this binding expects the library to export."""
    lib()
    return [n for n in dir(_lib) if n.startswith("tgv_")]


def _check(d, status: int, server=None):
    if status != TGV_OK:
        if server is not None:
            msg = lib().tgv_server_last_error(server).decode()
        else:
            msg = lib().tgv_last_error(d).decode() if d else ""
        raise TgvError(status, msg)


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def make_camera(cam) -> tgv_camera:
    c = tgv_camera()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, np.float64).reshape(9)
    C = np.asarray(cam.C, np.float64).reshape(3)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.C[k] = float(C[k])
    c.width, c.height, c.model = int(cam.width), int(cam.height), int(getattr(cam, "model", 0))
    return c


ITER_KERNELS = {"pipelined": 0, "one_brick_per_cta": 1, "paired": 2}


def make_params(nbins=8, alpha1=1.0, alpha0=2.0, lam=1.0, tau=0.2, sigma=0.2, storage="fp32", clamp_u=True,
                centres=0, box_v=2.0, iter_kernel="paired", x_run=0, hist_form="gather", wait_cycles=0,
                wait_test=0) -> tgv_params:
    p = tgv_params()
    _check(None, lib().tgv_default_params(ctypes.byref(p)))
    p.nbins, p.alpha1, p.alpha0, p.lam, p.tau, p.sigma = int(nbins), alpha1, alpha0, lam, tau, sigma
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.clamp_u, p.centres, p.box_v = int(bool(clamp_u)), int(centres), box_v
    p.iter_kernel = ITER_KERNELS[iter_kernel] if isinstance(iter_kernel, str) else int(iter_kernel)
    p.x_run = int(x_run)
    p.hist_form = HIST_FORMS[hist_form] if isinstance(hist_form, str) else int(hist_form)
    p.wait_cycles, p.wait_test = int(wait_cycles), int(wait_test)
    return p


# ------------------------------------------------------------------------------------ C entry points
def _fill_desc(d: tgv_level_desc, lv, keep: list):
    bc = _host(lv.bricks, np.int32).reshape(-1, 3)
    fr = getattr(lv, "frozen", None)
    fc = _host(fr, np.int32).reshape(-1, 3) if fr is not None else np.zeros((0, 3), np.int32)
    fu = getattr(lv, "frozen_u", None)
    fv = getattr(lv, "frozen_v", None)
    fu = _host(fu, np.float32) if (fu is not None and len(fc)) else None
    fv = _host(fv, np.float32) if (fv is not None and len(fc)) else None
    keep += [bc, fc, fu, fv]
    for a in range(3):
        d.origin[a] = float(np.asarray(lv.origin)[a])
    d.h = float(lv.h)
    d.radius = float(getattr(lv, "radius", 0.0) or 0.0)
    d.nbricks, d.brick_coords = bc.shape[0], _ptr(bc)
    d.nfrozen, d.frozen_coords = fc.shape[0], _ptr(fc) if len(fc) else None
    d.frozen_u, d.frozen_v = _ptr(fu), _ptr(fv)


def tgv_create_domain(levels, params: tgv_params, stream: int = 0):
    """levels: objects with origin, h, radius, bricks, frozen, frozen_u, frozen_v (synth.DomainDesc)."""
    keep = []
    descs = (tgv_level_desc * len(levels))()
    for k, lv in enumerate(levels):
        _fill_desc(descs[k], lv, keep)
    out = ctypes.c_void_p()
    st = lib().tgv_create_domain(descs, len(levels), ctypes.byref(params), ctypes.c_void_p(stream or 0),
                                 ctypes.byref(out))
    _check(None, st)
    del keep
    return out


def tgv_destroy_domain(d):
    lib().tgv_destroy_domain(d)


def tgv_accumulate_depthmaps(d, level: int, cams, depth, votes=None):
    """depth: CUDA tensor (nmaps, H, W) or (H, W) float32, contiguous rows."""
    if depth.dim() == 2:
        depth = depth.unsqueeze(0)
    nmaps, H, W = depth.shape
    arr = (tgv_camera * nmaps)(*[make_camera(c) for c in cams])
    vts = None if votes is None else np.ascontiguousarray(votes, np.uint32)
    st = lib().tgv_accumulate_depthmaps(d, level, arr, nmaps, depth.data_ptr(), depth.stride(1), depth.stride(0),
                                        _ptr(vts))
    _check(d, st)


def tgv_accumulate_depthmap(d, level: int, cam, depth, vote: int = 1):
    c = make_camera(cam)
    _check(d, lib().tgv_accumulate_depthmap(d, level, ctypes.byref(c), depth.data_ptr(), depth.stride(0), vote))


def tgv_solve(d, level: int, iterations: int, energy: bool = False):
    out = np.zeros(4) if energy else None
    _check(d, lib().tgv_solve(d, level, iterations, _ptr(out)))
    return out


def tgv_solve_graph(d, level: int, iterations: int, energy: bool = False):
    out = np.zeros(4) if energy else None
    _check(d, lib().tgv_solve_graph(d, level, iterations, _ptr(out)))
    return out


def tgv_solve_chunks(d, level: int, first, iterations, run_length: int = 0):
    """Persistent batched solve: chunk c = active bricks [first[c], first[c+1]) runs
    iterations[c] iterations (host arrays of nchunks + 1 int64 and nchunks int32)."""
    f = np.ascontiguousarray(first, dtype=np.int64)
    it = np.ascontiguousarray(iterations, dtype=np.int32)
    if f.size != it.size + 1:
        raise ValueError("first needs one entry more than iterations")
    _check(d, lib().tgv_solve_chunks(d, level, int(it.size), f.ctypes.data, it.ctypes.data, int(run_length)))


def tgv_set_work_list(d, level: int, bricks=None):
    """bricks: None (every active brick) or a host/device int32 array of brick indices."""
    if bricks is None:
        _check(d, lib().tgv_set_work_list(d, level, None, -1))
        return
    b = bricks if hasattr(bricks, "data_ptr") else _host(bricks, np.int32)
    _check(d, lib().tgv_set_work_list(d, level, _ptr(b), int(b.shape[0])))


def tgv_energy(d, level: int) -> np.ndarray:
    out = np.zeros(4)
    _check(d, lib().tgv_energy(d, level, _ptr(out)))
    return out


def tgv_energy_noalloc(nbricks: int, nall: int, u, v, p, q, hist, nbr, params: tgv_params, stream: int = 0,
                       out=None) -> np.ndarray:
    """Energy / dual / gap of a state held in caller-owned device buffers (no allocation).

    For callers that may not allocate device memory; u, v, p, q, hist, nbr are
    device tensors in the layout documented at tgv_state_view in include/tgv.h.
    Raises TgvError on a non-zero status.
    """
    view = tgv_state_view(int(nbricks), int(nall), _ptr(u), _ptr(v), _ptr(p), _ptr(q), _ptr(hist), _ptr(nbr))
    if out is None:
        out = np.zeros(4)
    st = lib().tgv_energy_noalloc(ctypes.byref(view), ctypes.byref(params), ctypes.c_void_p(stream or 0), _ptr(out))
    _check(None, st)
    return out



def tgv_extract_field(d, level: int, field: str, out=None):
    fid, nc = FIELDS[field]
    n = lib().tgv_level_voxels(d, level)
    if out is None:
        out = np.empty((n, nc), np.float32)
    _check(d, lib().tgv_extract_field(d, level, fid, _ptr(out), n * nc))
    return out


def tgv_set_field(d, level: int, field: str, values):
    fid, nc = FIELDS[field]
    n = lib().tgv_level_voxels(d, level)
    vals = values if hasattr(values, "data_ptr") else _host(values, np.float32)
    _check(d, lib().tgv_set_field(d, level, fid, _ptr(vals), n * nc))


def tgv_extract_histograms(d, level: int, nbins: int, out=None):
    n = lib().tgv_level_voxels(d, level)
    if out is None:
        out = np.empty((n, nbins), np.uint32)
    _check(d, lib().tgv_extract_histograms(d, level, _ptr(out), n * nbins))
    return out


def tgv_set_histograms(d, level: int, hist):
    h = hist if hasattr(hist, "data_ptr") else _host(hist, np.uint32)
    n = h.shape[0] * h.shape[1]
    _check(d, lib().tgv_set_histograms(d, level, _ptr(h), n))


def tgv_reset(d, level: int, clear_hist: bool = False):
    _check(d, lib().tgv_reset(d, level, int(clear_hist)))


def tgv_prolong(d, from_level: int):
    _check(d, lib().tgv_prolong(d, from_level))


def tgv_synchronize(d):
    _check(d, lib().tgv_synchronize(d))


def tgv_domain_bytes(d) -> int:
    return int(lib().tgv_domain_bytes(d))


def tgv_level_voxels(d, level: int) -> int:
    return int(lib().tgv_level_voxels(d, level))


def tgv_launch_count(d) -> int:
    return int(lib().tgv_launch_count(d))


def tgv_copy_mesh(d, verts: np.ndarray, tris: np.ndarray):
    """Copies the last extracted mesh into (nv, 3) float32 and (nt, 3) int32 host arrays."""
    _check(d, lib().tgv_copy_mesh(d, verts.ctypes.data, verts.shape[0], tris.ctypes.data, tris.shape[0]))


def tgv_extract_mesh(d, level: int):
    """Marching cubes of the level's u: (vertices (nv, 3) float32, triangles (nt, 3) int32)."""
    nv, nt = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(d, lib().tgv_extract_mesh(d, level, ctypes.byref(nv), ctypes.byref(nt)))
    verts = np.zeros((nv.value, 3), np.float32)
    tris = np.zeros((nt.value, 3), np.int32)
    tgv_copy_mesh(d, verts, tris)
    return verts, tris


def tgv_composite_create(d):
    h = ctypes.c_void_p()
    _check(d, lib().tgv_composite_create(d, ctypes.byref(h)))
    return h


def tgv_composite_solve(c, d, iterations: int):
    _check(d, lib().tgv_composite_solve(c, int(iterations)))


def tgv_composite_leaves(c) -> int:
    return int(lib().tgv_composite_leaves(c))


def tgv_composite_level_leaves(c, level: int) -> int:
    return int(lib().tgv_composite_level_leaves(c, level))


def tgv_composite_extract(c, d) -> np.ndarray:
    out = np.zeros(tgv_composite_leaves(c), np.float32)
    _check(d, lib().tgv_composite_extract(c, out.ctypes.data, out.size))
    return out


def tgv_composite_scatter(c, d):
    _check(d, lib().tgv_composite_scatter(c))


def tgv_composite_launch_count(c) -> int:
    return int(lib().tgv_composite_launch_count(c))


def tgv_composite_treetop(c, d, root_bits: int, max_cubes: int):
    """Treetop parts (Sec. 4.3): (depth, code, first, last) per part in Z-order and the
    part of every leaf (composite order)."""
    n = ctypes.c_int64(0)
    _check(d, lib().tgv_composite_treetop(c, int(root_bits), int(max_cubes), ctypes.byref(n)))
    return tgv_composite_treetop_parts(c, d, n.value)


def tgv_composite_treetop_parts(c, d, k: int):
    """The last treetop's k parts and the part of every leaf."""
    depth = np.zeros(k, np.int32)
    code = np.zeros(k, np.uint64)
    first = np.zeros(k, np.int64)
    last = np.zeros(k, np.int64)
    part = np.zeros(tgv_composite_leaves(c), np.int32)
    _check(d, lib().tgv_composite_treetop_parts(c, depth.ctypes.data, code.ctypes.data, first.ctypes.data,
                                                last.ctypes.data, part.ctypes.data))
    return depth, code, first, last, part


def tgv_composite_destroy(c):
    lib().tgv_composite_destroy(c)


class Composite:
    """Joint solve of every level of a Domain on their composite grid."""

    def __init__(self, dom: "Domain"):
        self.dom = dom
        self.handle = tgv_composite_create(dom.handle)

    @property
    def leaves(self):
        return tgv_composite_leaves(self.handle)

    def level_leaves(self, level):
        return tgv_composite_level_leaves(self.handle, level)

    def solve(self, iterations):
        tgv_composite_solve(self.handle, self.dom.handle, iterations)

    def u(self):
        return tgv_composite_extract(self.handle, self.dom.handle)

    def scatter(self):
        tgv_composite_scatter(self.handle, self.dom.handle)

    def treetop(self, root_bits, max_cubes):
        return tgv_composite_treetop(self.handle, self.dom.handle, root_bits, max_cubes)

    @property
    def launches(self):
        return tgv_composite_launch_count(self.handle)

    def close(self):
        if self.handle:
            tgv_composite_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class tgv_octree_cfg(ctypes.Structure):
    _fields_ = [("root_min", ctypes.c_double * 3), ("root_edge", ctypes.c_double), ("depth_min", ctypes.c_int32),
                ("depth_max", ctypes.c_int32), ("band", ctypes.c_int32)]


class OctreeLevel:
    """One level built by tgv_octree_build, shaped like a level description
    (origin, h, bricks, frozen) for tgv.Domain."""

    def __init__(self, origin, h, bricks, frozen):
        self.origin, self.h, self.bricks, self.frozen = np.asarray(origin), float(h), bricks, frozen
        self.frozen_u = self.frozen_v = None
        self.radius = 0.0

    @property
    def nbricks(self):
        return int(self.bricks.shape[0])

    @property
    def nvox(self):
        return 512 * self.nbricks

    @property
    def nfrozen(self):
        return int(self.frozen.shape[0])


def tgv_octree_levels(o) -> int:
    return int(lib().tgv_octree_levels(o))


def tgv_octree_samples(o) -> int:
    return int(lib().tgv_octree_samples(o))


def tgv_octree_level(o, level: int):
    """(nactive, nfrozen, origin (3,), h) of one built level."""
    na, nf, hh = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_double(0)
    org = (ctypes.c_double * 3)()
    _check(None, lib().tgv_octree_level(o, level, ctypes.byref(na), ctypes.byref(nf), org, ctypes.byref(hh)))
    return na.value, nf.value, np.array(org[:]), hh.value


def tgv_octree_bricks(o, level: int):
    """(active (na, 3), frozen (nf, 3)) int32 brick coordinates of one built level."""
    na, nf, _, _ = tgv_octree_level(o, level)
    act = np.zeros((na, 3), np.int32)
    frz = np.zeros((nf, 3), np.int32)
    _check(None, lib().tgv_octree_bricks(o, level, act.ctypes.data, frz.ctypes.data))
    return act, frz


def tgv_octree_destroy(o):
    lib().tgv_octree_destroy(o)


def tgv_octree_build(cams, depth, root_min, root_edge: float, depth_min: int, depth_max: int, band: int = 1,
                     stream: int = 0):
    """Brick levels from depth maps, pinhole or spherical (CUDA tensor (nmaps, H, W));
    returns (list of OctreeLevel, number of samples)."""
    if depth.dim() == 2:
        depth = depth.unsqueeze(0)
    nmaps = depth.shape[0]
    cfg = tgv_octree_cfg()
    for a in range(3):
        cfg.root_min[a] = float(root_min[a])
    cfg.root_edge, cfg.depth_min, cfg.depth_max, cfg.band = float(root_edge), int(depth_min), int(depth_max), int(band)
    arr = (tgv_camera * nmaps)(*[make_camera(c) for c in cams])
    h = ctypes.c_void_p()
    _check(None, lib().tgv_octree_build(ctypes.byref(cfg), arr, nmaps, depth.data_ptr(), depth.stride(1),
                                        depth.stride(0), ctypes.c_void_p(stream), ctypes.byref(h)))
    try:
        levels = []
        for l in range(tgv_octree_levels(h)):
            _, _, org, hh = tgv_octree_level(h, l)
            act, frz = tgv_octree_bricks(h, l)
            levels.append(OctreeLevel(org, hh, act, frz))
        return levels, tgv_octree_samples(h)
    finally:
        tgv_octree_destroy(h)


def tgv_pair_run_length(nbr: np.ndarray, work=None, slots: int = 296, storage="fp32") -> int:
    """Run length the paired kernel picks for a level with neighbour rows `nbr`
    ((nbricks, 12) int32, library layout) and an optional work list (host only)."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int32).reshape(-1, 12)
    w = None if work is None else np.ascontiguousarray(work, dtype=np.int32)
    out = ctypes.c_int32(0)
    _check(None, lib().tgv_pair_run_length(nbr.ctypes.data, nbr.shape[0], None if w is None else w.ctypes.data,
                                           0 if w is None else w.size, int(slots),
                                           STORAGE[storage] if isinstance(storage, str) else int(storage),
                                           ctypes.byref(out)))
    return int(out.value)


# ------------------------------------------------------------------------------------ convenience
class Domain:
    """Owns one tgv_domain handle; methods forward to the C entry points."""

    def __init__(self, levels, nbins=8, storage="fp32", stream: int = 0, **kw):
        """iter_kernel="auto" asks the autotuner (cached per size class) for the kernel form."""
        self.nbins = int(nbins)
        self.levels = list(levels)
        self.use_graph = False
        if kw.get("iter_kernel") == "auto":
            from . import autotune
            nvox = max(512 * int(np.asarray(lv.bricks).reshape(-1, 3).shape[0]) for lv in self.levels)
            rec = autotune.choose(storage, nbins, nvox)
            kw["iter_kernel"] = rec["iter_kernel"] if rec else "paired"
            self.use_graph = bool(rec and rec.get("graph"))
        self.params = make_params(nbins=nbins, storage=storage, **kw)
        self.handle = tgv_create_domain(self.levels, self.params, stream)

    def close(self):
        if self.handle:
            tgv_destroy_domain(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def accumulate(self, level, cams, depth, votes=None):
        tgv_accumulate_depthmaps(self.handle, level, cams, depth, votes)

    def solve(self, level, iterations, energy=False):
        if self.use_graph:
            return tgv_solve_graph(self.handle, level, iterations, energy)
        return tgv_solve(self.handle, level, iterations, energy)

    def energy(self, level=0):
        return tgv_energy(self.handle, level)

    def solve_graph(self, level, iterations, energy=False):
        return tgv_solve_graph(self.handle, level, iterations, energy)

    def set_work_list(self, level, bricks=None):
        tgv_set_work_list(self.handle, level, bricks)

    def solve_chunks(self, level, first, iterations, run_length=0):
        tgv_solve_chunks(self.handle, level, first, iterations, run_length)

    def field(self, level, name, out=None):
        return tgv_extract_field(self.handle, level, name, out)

    def mesh(self, level=0):
        return tgv_extract_mesh(self.handle, level)

    def set_field(self, level, name, values):
        tgv_set_field(self.handle, level, name, values)

    def histograms(self, level=0, out=None):
        return tgv_extract_histograms(self.handle, level, self.nbins, out)

    def set_histograms(self, level, hist):
        tgv_set_histograms(self.handle, level, hist)

    def reset(self, level, clear_hist=False):
        tgv_reset(self.handle, level, clear_hist)

    def prolong(self, from_level):
        tgv_prolong(self.handle, from_level)

    def synchronize(self):
        tgv_synchronize(self.handle)

    def voxels(self, level=0):
        return tgv_level_voxels(self.handle, level)

    @property
    def launches(self):
        return tgv_launch_count(self.handle)

    @property
    def nbytes(self):
        return tgv_domain_bytes(self.handle)


# ------------------------------------------------------------------------------------ serving
def tgv_server_create(capacity_bricks: int, capacity_frozen: int, params: tgv_params, stream: int,
                      staging_bytes: int = 0):
    cfg = tgv_server_cfg(int(capacity_bricks), int(capacity_frozen), int(staging_bytes))
    out = ctypes.c_void_p()
    _check(None, lib().tgv_server_create(ctypes.byref(cfg), ctypes.byref(params), ctypes.c_void_p(stream),
                                         ctypes.byref(out)))
    return out


def tgv_server_submit(s, chunk, hist, iterations: int) -> int:
    """chunk: DomainDesc-like (bricks, frozen, frozen_u, frozen_v); hist: (nvox, nbins) uint32 host/device."""
    keep = []
    d = tgv_level_desc()
    _fill_desc(d, chunk, keep)
    h = hist if hasattr(hist, "data_ptr") else _host(hist, np.uint32)
    t = ctypes.c_uint64()
    st = lib().tgv_server_submit(s, ctypes.byref(d), _ptr(h), int(iterations), ctypes.byref(t))
    _check(None, st, server=s)
    return int(t.value)


def tgv_server_step(s, max_iterations: int) -> int:
    f = ctypes.c_int32()
    _check(None, lib().tgv_server_step(s, int(max_iterations), ctypes.byref(f)), server=s)
    return int(f.value)


def tgv_server_poll(s, ticket: int) -> bool:
    f = ctypes.c_int32()
    _check(None, lib().tgv_server_poll(s, ctypes.c_uint64(ticket), ctypes.byref(f)), server=s)
    return bool(f.value)


def tgv_server_extract(s, ticket: int, nvox: int, out=None):
    if out is None:
        out = np.empty(nvox, np.float32)
    _check(None, lib().tgv_server_extract(s, ctypes.c_uint64(ticket), _ptr(out), int(nvox)), server=s)
    return out


def tgv_server_free_bricks(s) -> int:
    return int(lib().tgv_server_free_bricks(s))


def tgv_server_running(s) -> int:
    return int(lib().tgv_server_running(s))


def tgv_server_voxel_updates(s) -> int:
    return int(lib().tgv_server_voxel_updates(s))


def tgv_server_last_error(s) -> str:
    return lib().tgv_server_last_error(s).decode()


def tgv_server_synchronize(s):
    _check(None, lib().tgv_server_synchronize(s), server=s)


def tgv_server_destroy(s):
    lib().tgv_server_destroy(s)


class Server:
    """Owns one tgv_server handle; methods forward to the C entry points."""

    def __init__(self, capacity_bricks, capacity_frozen, nbins=8, storage="fp32", stream: int = 0,
                 staging_bytes: int = 0, **kw):
        self.params = make_params(nbins=nbins, storage=storage, **kw)
        self.handle = tgv_server_create(capacity_bricks, capacity_frozen, self.params, stream, staging_bytes)
        self.nvox = {}

    def close(self):
        if self.handle:
            tgv_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, chunk, hist, iterations):
        t = tgv_server_submit(self.handle, chunk, hist, iterations)
        self.nvox[t] = 512 * int(np.asarray(chunk.bricks).reshape(-1, 3).shape[0])
        return t

    def step(self, max_iterations):
        return tgv_server_step(self.handle, max_iterations)

    def done(self, ticket):
        return tgv_server_poll(self.handle, ticket)

    def extract(self, ticket, out=None):
        u = tgv_server_extract(self.handle, ticket, self.nvox[ticket], out)
        del self.nvox[ticket]
        return u

    @property
    def running(self):
        return tgv_server_running(self.handle)

    @property
    def free_bricks(self):
        return tgv_server_free_bricks(self.handle)

    @property
    def voxel_updates(self):
        return tgv_server_voxel_updates(self.handle)

    def synchronize(self):
        tgv_server_synchronize(self.handle)
