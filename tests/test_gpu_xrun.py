"""Runs of work items in the paired iteration kernel.

A CTA takes runs of consecutive work items; when the next item is the +x
neighbour brick, the x-face duals pass between the two on chip (the -x p halo
of the next brick, the parked x = 7 v update of this one) instead of being
recomputed.  The iteration (Eq. 2-3) is the same whichever way a dual reaches
its reader, so every field must be bit-identical for any run length and any
order of the work items; the oracle bounds the result as in the parity tests.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2107_14790_b300 import tgv

pytestmark = pytest.mark.gpu
FIELDS = ("u", "ubar", "v", "vbar", "p", "q")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2107_14790_b300 import build
    build.build()
    assert torch.cuda.is_available()
    tgv.lib()


def ragged_domain(seed, nx=7, ny=4, nz=3, drop=0.12, nfrozen=9):
    """x-rows of bricks with holes (runs break inside rows) and a few frozen bricks."""
    rng = np.random.default_rng(seed)
    box = np.array([(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)], np.int32)
    keep = rng.random(len(box)) > drop
    act, rest = box[keep], box[~keep]
    frz = rest[:nfrozen]
    fu = rng.uniform(-1, 1, (len(frz), 512)).astype(np.float32)
    fv = rng.normal(0, 0.1, (len(frz), 3, 512)).astype(np.float32)
    desc = synth.DomainDesc(np.zeros(3), 1.0, act, frozen=frz, frozen_u=fu, frozen_v=fv)
    return desc, synth.random_histograms(rng, desc.nvox, 10, max_count=15)


def run(desc, hist, iters, storage="fp32", x_run=0, work=None):
    with tgv.Domain([desc], nbins=10, storage=storage, stream=torch.cuda.current_stream().cuda_stream,
                    iter_kernel="paired", x_run=x_run) as dom:
        dom.set_histograms(0, hist)
        if work is not None:
            dom.set_work_list(0, work)
        dom.solve(0, iters)
        return {f: dom.field(0, f) for f in FIELDS}


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_run_length_does_not_change_any_field(storage):
    desc, hist = ragged_domain(5)
    ref = run(desc, hist, 29, storage, x_run=1)  # no hand-over: every halo recomputed
    for R in (2, 3, 7, 8, 64, 0):
        got = run(desc, hist, 29, storage, x_run=R)
        for f in FIELDS:
            np.testing.assert_array_equal(got[f], ref[f], err_msg=f"{storage} x_run={R} field {f}")
    if storage == "fp32":
        orc = oracle.OracleLevel(desc, 10)
        orc.hist[:] = hist
        orc.iterate(29)
        assert np.max(np.abs(ref["u"][:, 0] - orc.u)) <= 1e-4


def test_item_order_does_not_change_any_field():
    """A work list holding every brick, in row order, reversed and shuffled: hand-overs
    happen only where the next item is the +x neighbour; the fields never change."""
    desc, hist = ragged_domain(6, nx=9, ny=3, nz=2, nfrozen=4)
    ref = run(desc, hist, 17, x_run=1)
    nb = desc.nbricks
    orders = [np.arange(nb), np.arange(nb)[::-1], np.random.default_rng(3).permutation(nb)]
    for order in orders:
        for R in (4, 9):
            got = run(desc, hist, 17, x_run=R, work=np.ascontiguousarray(order, dtype=np.int32))
            for f in FIELDS:
                np.testing.assert_array_equal(got[f], ref[f])


def test_long_rows_dense_block():
    """A dense block whose x-rows are longer than the runs, with many runs per CTA."""
    nb = 12
    desc = synth.DomainDesc(np.zeros(3), 1.0 / (8 * nb), synth.dense_bricks(nb))
    hist = synth.random_histograms(np.random.default_rng(8), desc.nvox, 10, max_count=20)
    ref = run(desc, hist, 6, x_run=1)
    for R in (5, 8, 16, 0):
        got = run(desc, hist, 6, x_run=R)
        for f in FIELDS:
            np.testing.assert_array_equal(got[f], ref[f])


def test_run_length_is_validated():
    desc, hist = ragged_domain(5)
    for bad in (-1, 65):
        with pytest.raises(tgv.TgvError):
            run(desc, hist, 1, x_run=bad)
