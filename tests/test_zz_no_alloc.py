"""tgv_energy_noalloc against tgv_energy on the same state.

tgv_energy_noalloc serves callers that may not allocate device memory (a
serving process whose HBM is fully reserved for admitted requests, or a host
framework whose memory pool owns the device): they keep the state in their own
buffers and the library uses a fixed scratch array instead of cudaMalloc.
This file runs last (pytest collects it after the other test files) and also
passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

import synth
from paper_2107_14790_b300 import tgv

pytestmark = pytest.mark.gpu

SLOTS = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
         (-1, 1, 0), (-1, 0, 1), (1, -1, 0), (0, -1, 1), (1, 0, -1), (0, 1, -1)]


def layout_state(desc, u, v, p, q, hist, nbins, dtype):
    """Caller-owned device buffers in the tgv_state_view layout, built from voxel-major host arrays."""
    nb = desc.nbricks
    nf = desc.nfrozen
    ua = np.concatenate([u.reshape(nb, 512), desc.frozen_u.reshape(nf, 512)]) if nf else u.reshape(nb, 512)
    va = v.reshape(nb, 512, 3).transpose(0, 2, 1)
    if nf:
        va = np.concatenate([va, desc.frozen_v.reshape(nf, 3, 512)])
    pa = p.reshape(nb, 512, 3).transpose(0, 2, 1)
    qa = q.reshape(nb, 512, 6).transpose(0, 2, 1)
    npairs = (nbins + 1) // 2
    hp = np.zeros((nb, npairs, 512), np.uint32)
    h = hist.reshape(nb, 512, nbins)
    for k in range(npairs):
        lo = h[:, :, 2 * k]
        hi = h[:, :, 2 * k + 1] if 2 * k + 1 < nbins else np.zeros_like(lo)
        hp[:, k, :] = lo | (hi << 16)
    index = {tuple(c): i for i, c in enumerate(desc.bricks.tolist())}
    if nf:
        index.update({tuple(c): nb + i for i, c in enumerate(desc.frozen.tolist())})
    nbr = np.array([[index.get((c[0] + o[0], c[1] + o[1], c[2] + o[2]), -1) for o in SLOTS]
                    for c in desc.bricks.tolist()], np.int32)
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    return dict(u=dev(ua, np.float32), v=dev(va, np.float32).to(dtype), p=dev(pa, np.float32).to(dtype),
                q=dev(qa, np.float32).to(dtype), hist=dev(hp.view(np.int32), np.int32), nbr=dev(nbr, np.int32),
                nbricks=nb, nall=nb + nf)


@pytest.mark.parametrize("storage,dtype", [("fp32", torch.float32), ("bf16", torch.bfloat16)])
def test_noalloc_energy_matches_tgv_energy_twice(storage, dtype):
    from paper_2107_14790_b300 import build
    build.build()
    sp = synth.chunk_workload(seed=31, nchunks=1, min_vox=40 * 512, max_vox=40 * 512, nbins_range=(10, 10))[0]
    desc, nbins = sp.domain, sp.nbins
    rng = np.random.default_rng(12)
    n = desc.nvox
    u = rng.uniform(-1, 1, n).astype(np.float32)
    v = rng.normal(0, 0.2, (n, 3)).astype(np.float32)
    p = rng.normal(0, 0.4, (n, 3)).astype(np.float32)
    q = rng.normal(0, 0.4, (n, 6)).astype(np.float32)
    if storage != "fp32":  # both sides must see the same rounded values
        rnd = lambda a: torch.from_numpy(a).to(dtype).float().numpy()
        v, p, q = rnd(v), rnd(p), rnd(q)
    stream = torch.cuda.current_stream().cuda_stream
    with tgv.Domain([desc], nbins=nbins, storage=storage, stream=stream) as dom:
        dom.set_histograms(0, sp.hist)
        for name, arr in (("u", u), ("v", v), ("p", p), ("q", q)):
            dom.set_field(0, name, arr)
        ref = dom.energy(0)
        params = dom.params
    st = layout_state(desc, u, v, p, q, sp.hist, nbins, dtype)
    for call in range(2):
        got = tgv.tgv_energy_noalloc(st["nbricks"], st["nall"], st["u"], st["v"], st["p"], st["q"], st["hist"],
                                     st["nbr"], params, stream)
        for k in range(3):
            assert abs(got[k] - ref[k]) <= 1e-6 * abs(ref[0]), (call, k, got, ref)
        assert got[3] == ref[3]


def test_noalloc_empty_level():
    params = tgv.make_params(nbins=8)
    empty = tgv.tgv_energy_noalloc(0, 0, None, None, None, None, None, None, params)
    assert list(empty) == [0.0, 0.0, 0.0, 1.0]


def test_noalloc_energy_of_a_level_with_many_bricks():
    """69,696 bricks (35.7 M voxels, a 33 x 33 x 64 brick box): the scratch holds one set of
    partial sums per CTA of the energy kernel, not per brick, so any level fits."""
    from paper_2107_14790_b300 import build
    build.build()
    nx, ny, nz = 33, 33, 64
    desc = synth.DomainDesc(np.zeros(3), 1.0 / 512, synth.dense_bricks(nx, ny, nz))
    nb, n, nbins = desc.nbricks, desc.nvox, 8
    g = torch.Generator(device="cuda").manual_seed(5)
    u = torch.rand(n, device="cuda", generator=g) * 2 - 1
    v = torch.randn(n, 3, device="cuda", generator=g) * 0.2
    p = torch.randn(n, 3, device="cuda", generator=g) * 0.4
    q = torch.randn(n, 6, device="cuda", generator=g) * 0.4
    hist = torch.randint(0, 12, (n, nbins), device="cuda", generator=g, dtype=torch.int32)
    stream = torch.cuda.current_stream().cuda_stream
    with tgv.Domain([desc], nbins=nbins, stream=stream) as dom:
        dom.set_histograms(0, hist.cpu().numpy().astype(np.uint32))
        for name, arr in (("u", u[:, None]), ("v", v), ("p", p), ("q", q)):
            dom.set_field(0, name, arr.cpu().numpy())
        ref = dom.energy(0)
        params = dom.params
    # the tgv_state_view layout: [brick][component][512], histogram words [brick][pair][512]
    per_brick = lambda a, c: a.reshape(nb, 512, c).transpose(1, 2).contiguous()
    h = hist.reshape(nb, 512, nbins)
    hp = torch.stack([h[:, :, 2 * k] | (h[:, :, 2 * k + 1] << 16) for k in range(nbins // 2)], 1).contiguous()
    coords = desc.bricks
    grid = np.full((nx, ny, nz), -1, np.int64)
    grid[coords[:, 0], coords[:, 1], coords[:, 2]] = np.arange(nb)
    nbr = np.full((nb, 12), -1, np.int32)
    for k, o in enumerate(SLOTS):
        c = coords + np.array(o)
        ok = np.all((c >= 0) & (c < np.array([nx, ny, nz])), axis=1)
        nbr[ok, k] = grid[c[ok, 0], c[ok, 1], c[ok, 2]]
    got = tgv.tgv_energy_noalloc(nb, nb, u.contiguous(), per_brick(v, 3), per_brick(p, 3), per_brick(q, 6), hp,
                                 torch.from_numpy(nbr).cuda(), params, stream)
    assert nb > 65536
    for k in range(3):
        assert abs(got[k] - ref[k]) <= 1e-6 * abs(ref[0]), (k, got, ref)
    assert got[3] == ref[3]
