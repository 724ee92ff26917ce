"""The FX16 storage form: v, vbar in FP16; p, q in 16-bit fixed point scaled by the radii of
their projection balls (|p| <= alpha1, |q|_F <= alpha0 of Eq. 2's dual constraints).

* encoding: a value x of p (q) is stored as the integer round(x * 32767 / alpha1) (alpha0),
  clamped to [-32767, 32767], and read back as integer * alpha / 32767, each step rounded
  once in FP32 -- checked element by element through tgv_set_field / tgv_extract_field;
* the three kernel forms (paired, pipelined, one brick per CTA) each stay within the stated
  accuracy (5e-3) of the FP64 oracle on a chunk with a frozen shell, and within it of each
  other;
* a union level of chunks equals each chunk solved alone bit for bit, as in FP32;
* the server accepts the form and its results equal solo runs.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2107_14790_b300 import tgv
from paper_2107_14790_b300.batching import union_level

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2107_14790_b300 import build
    build.build()
    tgv.lib()


def _fx_expected(x, alpha):
    f = np.float32
    isc = f(32767.0) / f(alpha)
    dsc = f(alpha) / f(32767.0)
    i = np.clip(np.rint((x.astype(np.float32) * isc).astype(np.float32)), -32767, 32767)
    return (i.astype(np.float32) * dsc).astype(np.float32)


@pytest.mark.parametrize("alpha1,alpha0", [(1.0, 2.0), (0.7, 3.5)])
def test_fixed_point_encoding_through_the_field_calls(alpha1, alpha0):
    sp = synth.chunk_workload(81, 1, 6 * 512, 6 * 512, (10, 10))[0]
    n = sp.domain.nvox
    rng = np.random.default_rng(5)
    p = rng.uniform(-alpha1, alpha1, (n, 3)).astype(np.float32)
    q = rng.uniform(-alpha0, alpha0, (n, 6)).astype(np.float32)
    p[:7, 0] = [0.0, alpha1, -alpha1, alpha1 * 1.0001, -alpha1 * 5, 1e-9, alpha1 / 65534]  # edges, clamp
    with tgv.Domain([sp.domain], nbins=10, storage="fx16", alpha1=alpha1, alpha0=alpha0) as dom:
        dom.set_field(0, "p", p)
        dom.set_field(0, "q", q)
        gp, gq = dom.field(0, "p"), dom.field(0, "q")
        v = rng.normal(0, 0.3, (n, 3)).astype(np.float32)
        dom.set_field(0, "v", v)
        gv = dom.field(0, "v")
    np.testing.assert_array_equal(gp, _fx_expected(p, alpha1))
    np.testing.assert_array_equal(gq, _fx_expected(q, alpha0))
    np.testing.assert_array_equal(gv, v.astype(np.float16).astype(np.float32))
    # inside the ball the error is half a step, plus the FP32 rounding of the two scales
    # and of the products (a few ulps of alpha)
    inside = np.abs(p) <= alpha1
    assert np.abs(gp - p)[inside].max() <= alpha1 / 65534 + 4 * 2.0 ** -24 * alpha1


def _chunk(seed=82, lo=20, hi=60):
    return synth.chunk_workload(seed, 1, lo * 512, hi * 512, (10, 10))[0]


def test_kernel_forms_meet_the_stated_accuracy():
    sp = _chunk()
    iters = 150
    o = oracle.OracleLevel(sp.domain, 10)
    o.hist[:] = sp.hist
    o.iterate(iters)
    s = torch.cuda.Stream()
    us = {}
    for form in ("paired", "pipelined", "one_brick_per_cta"):
        with tgv.Domain([sp.domain], nbins=10, storage="fx16", stream=s.cuda_stream, iter_kernel=form) as dom:
            dom.set_histograms(0, sp.hist)
            dom.solve(0, iters)
            us[form] = dom.field(0, "u")[:, 0]
        err = np.abs(us[form] - o.u).max()
        print(f"fx16 {form}: max |du| vs oracle = {err:.3e}")
        assert err <= 5e-3
    assert np.abs(us["paired"] - us["pipelined"]).max() <= 5e-3
    assert np.abs(us["paired"] - us["one_brick_per_cta"]).max() <= 5e-3


@pytest.mark.parametrize("nbins", [8, 12, 5])
def test_paired_kernel_bin_counts_meet_the_stated_accuracy(nbins):
    """The paired kernel is compiled per bin count (8, 10 and 12; others read the count at
    run time), its FX16 step-unit arithmetic with it: each form within the stated accuracy
    (5e-3) of the FP64 oracle on a chunk with a frozen shell."""
    sp = synth.chunk_workload(85 + nbins, 1, 20 * 512, 40 * 512, (nbins, nbins))[0]
    iters = 100
    o = oracle.OracleLevel(sp.domain, nbins)
    o.hist[:] = sp.hist
    o.iterate(iters)
    s = torch.cuda.Stream()
    with tgv.Domain([sp.domain], nbins=nbins, storage="fx16", stream=s.cuda_stream) as dom:
        dom.set_histograms(0, sp.hist)
        dom.solve(0, iters)
        u = dom.field(0, "u")[:, 0]
    err = np.abs(u - o.u).max()
    print(f"fx16 paired, {nbins} bins: max |du| vs oracle = {err:.3e}")
    assert err <= 5e-3


def test_union_level_equals_each_chunk_alone():
    specs = synth.chunk_workload(83, 3, 6 * 512, 40 * 512, (10, 10))
    U = union_level([sp.domain for sp in specs])
    s = torch.cuda.Stream()
    with tgv.Domain([U], nbins=10, storage="fx16", stream=s.cuda_stream) as dom:
        dom.set_histograms(0, np.concatenate([sp.hist for sp in specs]))
        dom.solve(0, 25)
        u = dom.field(0, "u")[:, 0]
    for sp, (a, b) in zip(specs, U.ranges):
        with tgv.Domain([sp.domain], nbins=10, storage="fx16", stream=s.cuda_stream) as dom:
            dom.set_histograms(0, sp.hist)
            dom.solve(0, 25)
            np.testing.assert_array_equal(u[512 * a:512 * b], dom.field(0, "u")[:, 0])


def test_server_with_fixed_point_duals_equals_solo_runs():
    specs = synth.chunk_workload(84, 3, 6 * 512, 30 * 512, (10, 10))
    iters = [11, 20, 7]
    s = torch.cuda.Stream()
    cap = sum(sp.domain.nbricks for sp in specs)
    capf = sum(sp.domain.nfrozen for sp in specs)
    with tgv.Server(cap, capf, nbins=10, storage="fx16", stream=s.cuda_stream) as srv:
        t = [srv.submit(sp.domain, sp.hist, it) for sp, it in zip(specs, iters)]
        for _ in range(10):
            if all(srv.done(x) for x in t):
                break
            srv.step(100)
        got = [srv.extract(x) for x in t]
    for sp, it, u in zip(specs, iters, got):
        with tgv.Domain([sp.domain], nbins=10, storage="fx16", stream=s.cuda_stream) as dom:
            dom.set_histograms(0, sp.hist)
            dom.solve(0, it)
            np.testing.assert_array_equal(u, dom.field(0, "u")[:, 0])
