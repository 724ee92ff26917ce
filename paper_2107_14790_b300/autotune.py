"""Autotuner for the fused iteration: picks the kernel form per (storage, bins, size class).

Candidates are the three forms of the fused iteration kernel (paired /
pipelined / one brick per CTA: they differ in warps per brick, voxels per
thread and whether bricks are streamed through shared memory) crossed with
plain launches or CUDA-graph replay.  Each candidate is timed with CUDA events
on a seeded dense domain of the size class's representative size; the winner
is cached in a JSON file keyed by device name, storage, bin count and size
class, so later domains of that class reuse it without timing.

Cache file: $TGV_AUTOTUNE_CACHE, else autotune_cache.json next to this module.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Optional

import numpy as np

from . import tgv

FORMS = ("paired", "pipelined", "one_brick_per_cta")
# active-voxel size classes: upper bound (exclusive) -> representative dense edge in voxels
SIZE_CLASSES = [(1 << 18, 48), (1 << 21, 96), (1 << 24, 192), (1 << 62, 256)]
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("TGV_AUTOTUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json"))


def size_class(nvox: int) -> int:
    for k, (hi, _) in enumerate(SIZE_CLASSES):
        if nvox < hi:
            return k
    return len(SIZE_CLASSES) - 1


def _key(device: str, storage: str, nbins: int, cls: int) -> str:
    return f"{device}|{storage}|{nbins}|{cls}"


def _load() -> Dict[str, dict]:
    p = cache_path()
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except (OSError, ValueError):
            return {}
    return {}


def _store(cache: Dict[str, dict]):
    p = cache_path()
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def time_candidate(edge: int, nbins: int, storage: str, form: str, graph: bool, iters: int = 16,
                   seed: int = 11) -> float:
    """Microseconds per fused iteration on a dense edge^3 domain with seeded random histograms."""
    import torch
    import synth
    nb = max(1, edge // 8)
    desc = synth.DomainDesc(np.zeros(3), 1.0 / (8 * nb), synth.dense_bricks(nb))
    hist = synth.random_histograms(np.random.default_rng(seed), desc.nvox, nbins, max_count=20)
    stream = torch.cuda.Stream()
    with tgv.Domain([desc], nbins=nbins, storage=storage, stream=stream.cuda_stream, iter_kernel=form) as dom:
        dom.set_histograms(0, hist)
        run = dom.solve_graph if graph else dom.solve
        run(0, iters)  # warm up (and capture, for graphs)
        run(0, iters)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run(0, iters)
        e1.record(stream)
        dom.synchronize()
        return e0.elapsed_time(e1) * 1e3 / iters


def tune(storage: str, nbins: int, cls: int, force: bool = False) -> dict:
    """Times every candidate for one size class (unless cached) and returns the winner's record."""
    with _lock:
        cache = _load()
        key = _key(_device_name(), storage, nbins, cls)
        if key in cache and not force:
            return cache[key]
        edge = SIZE_CLASSES[cls][1]
        times = {}
        for form in FORMS:
            for graph in (False, True):
                times[f"{form}/{'graph' if graph else 'plain'}"] = time_candidate(edge, nbins, storage, form, graph)
        best = min(times, key=times.get)
        form, mode = best.split("/")
        rec = {"iter_kernel": form, "graph": mode == "graph", "us_per_iteration": times[best],
               "edge": edge, "candidates": times}
        cache[key] = rec
        _store(cache)
        return rec


def choose(storage: str, nbins: int, nvox: int, allow_tuning: bool = True) -> Optional[dict]:
    """Cached choice for a domain of `nvox` active voxels (tunes the class first if allowed)."""
    cls = size_class(nvox)
    try:
        key = _key(_device_name(), storage, nbins, cls)
    except Exception:
        return None
    rec = _load().get(key)
    if rec is None and allow_tuning:
        rec = tune(storage, nbins, cls)
    return rec


# ------------------------------------------------------------------------ the batched solve
# Candidates for a mix of chunks (one union level): the union form (one launch per iteration,
# replayed as a CUDA graph) with the paired kernel at several run lengths or the pipelined
# kernel (one voxel per thread, 512 threads: another CTA shape), and the persistent launch
# (tgv_solve_chunks) at several run lengths.
BATCH_CANDIDATES = ([("union_graph", "paired", x) for x in (0, 1, 4, 16)] + [("union_graph", "pipelined", 0)] +
                    [("persistent", "paired", r) for r in (8, 16, 32)])


def mix_signature(sizes) -> str:
    """Size classes of a chunk mix: counts of chunks per power-of-two voxel count."""
    cls = {}
    for n in sizes:
        k = int(np.log2(max(int(n), 1)))
        cls[k] = cls.get(k, 0) + 1
    return ",".join(f"{k}:{cls[k]}" for k in sorted(cls))


def sample_chunks(chunks, max_voxels: int = 8 << 20):
    """A sample of a chunk mix that keeps its size distribution: chunks taken at even steps
    through the size-sorted list until `max_voxels` voxels are reached (at least one)."""
    order = sorted(range(len(chunks)), key=lambda k: chunks[k].nvox)
    out, tot = [], 0
    step = max(1, len(order) // 16)
    for i in list(range(0, len(order), step)) + list(range(1, len(order), step)):
        c = chunks[order[i]]
        if out and tot + c.nvox > max_voxels:
            continue
        out.append(c)
        tot += c.nvox
    return out


def time_batch_candidate(U, hist, nbins: int, storage: str, cand, iters: int = 24) -> float:
    """Nanoseconds per voxel-iteration of one candidate on union level U with counts `hist`."""
    import torch
    form, kernel, x = cand
    stream = torch.cuda.Stream()
    kw = dict(iter_kernel=kernel, x_run=x if form == "union_graph" else 0)
    with tgv.Domain([U], nbins=nbins, storage=storage, stream=stream.cuda_stream, **kw) as dom:
        dom.set_histograms(0, hist)
        first = U.first
        its = [iters] * len(U.ranges)

        def run():
            if form == "union_graph":
                dom.solve_graph(0, iters)
            else:
                dom.solve_chunks(0, first, its, run_length=x)
        run()  # warm up and capture
        run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        dom.synchronize()
        return e0.elapsed_time(e1) * 1e6 / (iters * 512 * len(U.bricks))


def tune_batch(chunks, nbins: int, storage: str, hist_of=None, force: bool = False, seed: int = 12) -> dict:
    """Measures every batched candidate on a sample of the chunk mix it will serve and caches
    the fastest per (device, storage, bins, size classes of the mix).  `chunks`: DomainDesc-
    like chunks (bricks, frozen shell); `hist_of(chunk)` gives a chunk's counts (seeded
    random counts when None).  Returns the record: form, kernel, run length, ns per
    voxel-iteration and every candidate's time."""
    import synth
    from .batching import GROUP_VOXELS, union_level
    with _lock:
        cache = _load()
        key = f"batch|{_device_name()}|{storage}|{nbins}|{mix_signature([c.nvox for c in chunks])}"
        if key in cache and not force:
            return cache[key]
        sample = sample_chunks(chunks)
        U = union_level(sample)
        rng = np.random.default_rng(seed)
        def counts(c):
            if hist_of is None:
                return synth.random_histograms(rng, c.nvox, nbins, max_count=20)
            x = hist_of(c)
            return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
        hs = [counts(c) for c in sample]
        hist = np.concatenate(hs).astype(np.uint32)
        times = {}
        for cand in BATCH_CANDIDATES:
            times["/".join(map(str, cand))] = time_batch_candidate(U, hist, nbins, storage, cand)
        best = min(times, key=times.get)
        form, kernel, x = best.split("/")
        # group size of the union levels (batching.GROUP_VOXELS): measured on whole c4-style
        # mixes, where the effect shows; the sample here is smaller than one group
        rec = {"form": form, "iter_kernel": kernel, "run_length": int(x), "group_voxels": GROUP_VOXELS,
               "ns_per_voxel_iteration": times[best],
               "sample_chunks": len(sample), "sample_voxels": int(sum(c.nvox for c in sample)),
               "candidates": times}
        cache[key] = rec
        _store(cache)
        return rec
