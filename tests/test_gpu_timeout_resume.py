"""Failure detection of the bounded device-side waits, and checkpoint / resume.

Timeout: the paired kernel's CTAs wait (bounded) for the bulk copies that bring each
brick into shared memory.  With `wait_test = 1` every CTA's first wait targets a barrier
that nothing ever completes, so it runs out after `wait_cycles` (here about 0.1 ms):
no fault, no trap, no endless loop.  The CTA then sets the domain's error flag, waits
for its own copies in flight with the default budget and returns.  The next call that
synchronises reports TGV_ERR_TIMEOUT, every later call on that domain TGV_ERR_STATE,
and the CUDA context stays usable for other domains.

Checkpoint / resume: a level's whole iteration state (u, ubar, v, vbar, p, q) read back
after N1 iterations and loaded into a new domain continues exactly like the
uninterrupted run: after N1 + N2 iterations every field is equal bit for bit (the
ping-pong copy a field lives in is internal to the library; the ABI reads and writes
the current one).
"""
import numpy as np
import pytest
import torch

import synth
from paper_2107_14790_b300 import tgv

pytestmark = pytest.mark.gpu
FIELDS = ("u", "ubar", "v", "vbar", "p", "q")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2107_14790_b300 import build
    build.build()
    tgv.lib()


def chunk(seed=71, lo=30, hi=60, nbins=10):
    return synth.chunk_workload(seed, 1, lo * 512, hi * 512, (nbins, nbins))[0]


def test_a_wait_that_runs_out_reports_timeout_and_the_domain_stays_broken():
    sp = chunk()
    s = torch.cuda.Stream()
    with tgv.Domain([sp.domain], nbins=10, stream=s.cuda_stream, wait_cycles=200_000, wait_test=1) as dom:
        dom.set_histograms(0, sp.hist)
        dom.solve(0, 2)  # queued; nothing synchronises yet
        with pytest.raises(tgv.TgvError) as e:
            dom.synchronize()
        assert e.value.status == 5  # TGV_ERR_TIMEOUT
        assert "wait" in str(e.value)
        for call in (lambda: dom.solve(0, 1), lambda: dom.energy(0), lambda: dom.field(0, "u"),
                     lambda: dom.synchronize()):
            with pytest.raises(tgv.TgvError) as e:
                call()
            assert e.value.status == 6  # TGV_ERR_STATE
    # the context is still usable: a normal domain on the same stream solves as before
    ref = None
    for wait_cycles in (0, 50_000_000):  # default budget, and a stated one that suffices
        with tgv.Domain([sp.domain], nbins=10, stream=s.cuda_stream, wait_cycles=wait_cycles) as dom:
            dom.set_histograms(0, sp.hist)
            dom.solve(0, 9)
            dom.synchronize()
            u = dom.field(0, "u")
        if ref is None:
            ref = u
        np.testing.assert_array_equal(u, ref)
    assert np.abs(ref).max() > 0


def test_bad_wait_parameters_are_rejected():
    sp = chunk(72, 4, 4)
    for kw in (dict(wait_cycles=-1), dict(wait_test=2)):
        with pytest.raises(tgv.TgvError) as e:
            tgv.Domain([sp.domain], nbins=10, **kw)
        assert e.value.status == 1


@pytest.mark.parametrize("storage", ["fp32", "fp16", "fx16"])
@pytest.mark.parametrize("n1,n2", [(13, 17), (8, 5)])
def test_checkpoint_resume_is_bit_identical(storage, n1, n2):
    sp = chunk(73)
    s = torch.cuda.Stream()
    with tgv.Domain([sp.domain], nbins=10, storage=storage, stream=s.cuda_stream) as dom:
        dom.set_histograms(0, sp.hist)
        dom.solve(0, n1 + n2)
        want = {f: dom.field(0, f) for f in FIELDS}
    with tgv.Domain([sp.domain], nbins=10, storage=storage, stream=s.cuda_stream) as dom:
        dom.set_histograms(0, sp.hist)
        dom.solve(0, n1)
        ck = {f: dom.field(0, f) for f in FIELDS}
        hist = dom.histograms(0)
    with tgv.Domain([sp.domain], nbins=10, storage=storage, stream=s.cuda_stream) as dom:
        dom.set_histograms(0, hist)
        for f in FIELDS:
            dom.set_field(0, f, ck[f])
        dom.solve(0, n2)
        got = {f: dom.field(0, f) for f in FIELDS}
    for f in FIELDS:
        np.testing.assert_array_equal(got[f], want[f], err_msg=f)
