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


# ------------------------------------------------------------------ the persistent batched form
FIELDS = ("u", "ubar", "v", "vbar", "p", "q")


def solo(sp, iters, storage="fp32", **kw):
    s = torch.cuda.Stream()
    with tgv.Domain([sp.domain], nbins=sp.nbins, storage=storage, stream=s.cuda_stream, **kw) as dom:
        dom.set_histograms(0, sp.hist)
        dom.solve(0, iters)
        return {f: dom.field(0, f) for f in FIELDS}


def split(fields, U, k):
    a, b = U.ranges[k]
    return {f: v[512 * a:512 * b] for f, v in fields.items()}


@pytest.mark.parametrize("storage", ["fp32", "fx16", "fp16", "bf16"])
def test_persistent_launch_equals_solo_runs_and_the_oracle(storage):
    """Five uneven chunks with frozen shells and their own iteration counts (both parities)
    in one persistent launch: every field of every chunk equals the chunk solved alone,
    bit for bit, and u is within the form's bar of the oracle (FP32 1e-4, FX16 and FP16
    5e-3; BF16, which misses the stated accuracy, 1e-1)."""
    specs = synth.chunk_workload(63, 5, 4 * 512, 90 * 512, (10, 10), (ITERS, ITERS))
    iters = [ITERS, 37, ITERS - 1, 80, 1]
    U = union_level([sp.domain for sp in specs])
    s = torch.cuda.Stream()
    with tgv.Domain([U], nbins=10, storage=storage, stream=s.cuda_stream) as dom:
        dom.set_histograms(0, np.concatenate([sp.hist for sp in specs]))
        l0 = dom.launches
        dom.solve_chunks(0, U.first, iters)
        launches = dom.launches - l0
        got = {f: dom.field(0, f) for f in FIELDS}
    assert launches <= 2  # the persistent kernel (and the copy that aligns the parities)
    bar = {"fp32": 1e-4, "fx16": 5e-3, "fp16": 5e-3, "bf16": 1e-1}[storage]
    for k, sp in enumerate(specs):
        want = solo(sp, iters[k], storage)
        mine = split(got, U, k)
        for f in FIELDS:
            np.testing.assert_array_equal(mine[f], want[f], err_msg=f"chunk {k} field {f}")
        err = np.abs(mine["u"][:, 0] - oracle_u(sp, iters[k])).max()
        assert err <= bar, f"chunk {k}: max |du| = {err:.2e}"


@pytest.mark.parametrize("run_length", [1, 3, 16, 64])
def test_persistent_results_do_not_depend_on_the_run_length(run_length):
    specs = synth.chunk_workload(64, 4, 6 * 512, 60 * 512, (8, 8), (20, 20))
    U = union_level([sp.domain for sp in specs])
    s = torch.cuda.Stream()
    with tgv.Domain([U], nbins=8, stream=s.cuda_stream) as dom:
        dom.set_histograms(0, np.concatenate([sp.hist for sp in specs]))
        dom.solve_chunks(0, U.first, [20, 13, 20, 6], run_length=run_length)
        u = dom.field(0, "u")[:, 0]
    for k, (sp, it) in enumerate(zip(specs, [20, 13, 20, 6])):
        a, b = U.ranges[k]
        np.testing.assert_array_equal(u[512 * a:512 * b], solo(sp, it)["u"][:, 0])


def test_persistent_graph_replay_and_continuation():
    """The second identical call replays the captured graph; a plain solve continues
    from the state the persistent launch leaves (one current ping-pong copy)."""
    specs = synth.chunk_workload(65, 3, 6 * 512, 40 * 512, (10, 10), (10, 10))
    U = union_level([sp.domain for sp in specs])
    s = torch.cuda.Stream()
    with tgv.Domain([U], nbins=10, stream=s.cuda_stream) as dom:
        dom.set_histograms(0, np.concatenate([sp.hist for sp in specs]))
        dom.solve_chunks(0, U.first, [6, 6, 6])  # captured
        dom.solve_chunks(0, U.first, [6, 6, 6])  # same plan, same ping-pong copy: replayed
        dom.solve_chunks(0, U.first, [7, 7, 7])  # a new plan; the copy flips
        dom.solve_chunks(0, U.first, [5, 8, 3])  # mixed parities: the copy that aligns them runs
        dom.solve(0, 5)
        got = {f: dom.field(0, f) for f in FIELDS}
    for k, sp in enumerate(specs):
        want = solo(sp, 6 + 6 + 7 + [5, 8, 3][k] + 5)
        mine = split(got, U, k)
        for f in FIELDS:
            np.testing.assert_array_equal(mine[f], want[f], err_msg=f"chunk {k} field {f}")


def test_persistent_rejects_linked_chunks_and_work_lists():
    specs = synth.chunk_workload(66, 2, 8 * 512, 20 * 512, (10, 10))
    U = union_level([sp.domain for sp in specs])
    with tgv.Domain([U], nbins=10) as dom:
        a, b = U.ranges[0]
        with pytest.raises(tgv.TgvError) as e:  # a cut inside one chunk splits linked bricks
            dom.solve_chunks(0, [a, a + 1, U.ranges[1][1]], [3, 3])
        assert e.value.status == 1
        with pytest.raises(tgv.TgvError) as e:
            dom.solve_chunks(0, [a, a], [3])  # empty chunk
        assert e.value.status == 1
        dom.set_work_list(0, np.arange(a, b, dtype=np.int32))
        with pytest.raises(tgv.TgvError) as e:
            dom.solve_chunks(0, U.first, [3, 3])
        assert e.value.status == 1


def test_persistent_barrier_wait_that_runs_out_reports_timeout():
    specs = synth.chunk_workload(67, 2, 8 * 512, 20 * 512, (10, 10))
    U = union_level([sp.domain for sp in specs])
    s = torch.cuda.Stream()
    with tgv.Domain([U], nbins=10, stream=s.cuda_stream, wait_cycles=200_000, wait_test=1) as dom:
        dom.set_histograms(0, np.concatenate([sp.hist for sp in specs]))
        dom.solve_chunks(0, U.first, [4, 4])
        with pytest.raises(tgv.TgvError) as e:
            dom.synchronize()
        assert e.value.status == 5
        with pytest.raises(tgv.TgvError) as e:
            dom.solve_chunks(0, U.first, [4, 4])
        assert e.value.status == 6
