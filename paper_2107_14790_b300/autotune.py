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
