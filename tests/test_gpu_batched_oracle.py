"""The batched form against the oracle (Sec. 4.3 parts with the frozen border of Sec. 4.5).

Several chunks of uneven size, each a box of bricks wrapped in a frozen one-brick shell,
share one union level; one fused launch per iteration advances all of them (plain
launches, and the same launches replayed as a CUDA graph).  Each chunk is an independent
problem, so the oracle solves each alone, in FP64, and every chunk's u must lie within
1e-4 of it after the configured iterations (the FP32 bar of the single-domain tests).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2107_14790_b300 import tgv
from paper_2107_14790_b300.batching import union_level

pytestmark = pytest.mark.gpu
ITERS = 120


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2107_14790_b300 import build
    build.build()
    tgv.lib()


def oracle_u(sp, iters):
    o = oracle.OracleLevel(sp.domain, sp.nbins)
    o.hist[:] = sp.hist
    o.iterate(iters)
    return o.u


@pytest.mark.parametrize("nbins,seed", [(10, 61), (8, 62)])
@pytest.mark.parametrize("graph", [False, True])
def test_union_of_uneven_chunks_matches_the_oracle(nbins, seed, graph):
    # five chunks from 4 to 90 bricks, boxes of different shapes, frozen face shells
    specs = synth.chunk_workload(seed, 5, 4 * 512, 90 * 512, (nbins, nbins), (ITERS, ITERS))
    sizes = [sp.domain.nbricks for sp in specs]
    assert max(sizes) >= 4 * min(sizes)  # uneven
    assert all(sp.domain.nfrozen > 0 for sp in specs)
    U = union_level([sp.domain for sp in specs])
    hist = np.concatenate([sp.hist for sp in specs])
    s = torch.cuda.Stream()
    with tgv.Domain([U], nbins=nbins, stream=s.cuda_stream) as dom:
        dom.set_histograms(0, hist)
        if graph:
            dom.solve_graph(0, ITERS // 2)
            dom.solve_graph(0, ITERS // 2)  # replay
        else:
            dom.solve(0, ITERS)
        u = dom.field(0, "u")[:, 0]
    for k, sp in enumerate(specs):
        a, b = U.ranges[k]
        want = oracle_u(sp, ITERS)
        assert np.abs(want).max() > 0.1
        err = np.abs(u[512 * a:512 * b] - want).max()
        assert err <= 1e-4, f"chunk {k} ({sp.domain.nbricks} bricks): max |du| = {err:.2e}"
