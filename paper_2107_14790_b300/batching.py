"""Host orchestration of the batched and served forms (no arithmetic of the method).

* `union_level`: several independent chunks (Sec. 4.3 parts, each with its
  frozen border, Sec. 4.5) placed far apart in one brick level, so one launch
  of the fused iteration advances all of them;
* `RequestStream`: a request loop over `tgv.Server` objects (one per bin
  count) with arrival times, FIFO admission under the servers' fixed arena
  budget, rounds of `step` iterations and per-request latency.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import tgv



@dataclass
class UnionLevel:
    origin: np.ndarray
    h: float
    bricks: np.ndarray
    frozen: Optional[np.ndarray]
    frozen_u: Optional[np.ndarray]
    frozen_v: Optional[np.ndarray]
    ranges: List[tuple]  # active-brick range [a, b) of each chunk
    radius: float = 0.0

    @property
    def first(self) -> np.ndarray:
        """Brick ranges as the first-brick table of tgv_solve_chunks (nchunks + 1 entries)."""
        return np.array([a for a, _ in self.ranges] + [self.ranges[-1][1]], np.int64)


def union_level(domains: Sequence) -> UnionLevel:
    """One level holding every chunk of `domains` (DomainDesc-like): the chunks are laid
    side by side along x with a gap of two bricks between their extents (frozen shells
    included), so no face or edge link crosses chunks."""
    act, frz, fu, fv, ranges = [], [], [], [], []
    o = 0
    x_next = -(1 << 18)
    for c, dm in enumerate(domains):
        b = np.asarray(dm.bricks, np.int32).reshape(-1, 3)
        allb = b if getattr(dm, "frozen", None) is None or not len(dm.frozen) else \
            np.concatenate([b, np.asarray(dm.frozen, np.int32).reshape(-1, 3)])
        lo, hi = int(allb[:, 0].min()), int(allb[:, 0].max())
        shift = np.array([x_next - lo, 0, 0], np.int32)
        x_next += hi - lo + 3
        act.append(b + shift)
        ranges.append((o, o + b.shape[0]))
        o += b.shape[0]
        if getattr(dm, "frozen", None) is not None and len(dm.frozen):
            f = np.asarray(dm.frozen, np.int32).reshape(-1, 3)
            frz.append(f + shift)
            fu.append(np.asarray(dm.frozen_u, np.float32).reshape(-1, 512) if dm.frozen_u is not None
                      else np.zeros((f.shape[0], 512), np.float32))
            fv.append(np.asarray(dm.frozen_v, np.float32).reshape(-1, 3, 512) if dm.frozen_v is not None
                      else np.zeros((f.shape[0], 3, 512), np.float32))
    if x_next >= (1 << 19):
        raise ValueError("chunks do not fit the brick coordinate range of one level")
    return UnionLevel(np.asarray(domains[0].origin, np.float64), float(domains[0].h), np.concatenate(act),
                      np.concatenate(frz) if frz else None, np.concatenate(fu) if fu else None,
                      np.concatenate(fv) if fv else None, ranges)


@dataclass
class Request:
    rid: int
    chunk: object          # DomainDesc-like
    nbins: int
    iterations: int
    arrival: float         # seconds after the stream starts
    make_hist: Callable    # () -> (nvox, nbins) counts (host or device); called at admission
    hist: object = None
    ticket: int = 0
    admitted: float = -1.0
    finished: float = -1.0
    u: object = None


@dataclass
class StreamResult:
    latencies: np.ndarray
    wait: np.ndarray
    makespan: float
    voxel_updates: int
    completed: int
    max_running: int
    rounds: int
    requests: List[Request] = field(default_factory=list)


class RequestStream:
    """Runs requests through one server per bin count.

    Each round: admit arrived requests in arrival order while their server has
    room (BUDGET leaves a request queued), queue `round_iters` iterations on
    every server with running requests, then extract the requests the
    previous round finished.  Two rounds are kept in flight so the host work
    of one overlaps the device work of the other.
    """

    def __init__(self, servers: Dict[int, "tgv.Server"], streams: Dict[int, object], round_iters: int = 10,
                 keep_results: bool = False):
        self.servers = servers
        self.streams = streams
        self.round_iters = int(round_iters)
        self.keep = keep_results

    def run(self, requests: List[Request], clock=time.perf_counter) -> StreamResult:
        import torch

        reqs = sorted(requests, key=lambda r: r.arrival)
        vu0 = sum(srv.voxel_updates for srv in self.servers.values())
        pending = deque()
        running: Dict[int, Request] = {}
        nxt = 0
        done = 0
        rounds = 0
        max_running = 0
        t0 = clock()
        in_flight = []  # events of the previous round, with the tickets that round finished
        finishing = set()
        while done < len(reqs):
            now = clock() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            # admission, first come first served per server
            blocked = set()
            keep = deque()
            while pending:
                r = pending.popleft()
                if r.nbins in blocked:
                    keep.append(r)
                    continue
                if r.hist is None:
                    r.hist = r.make_hist()
                try:
                    r.ticket = self.servers[r.nbins].submit(r.chunk, r.hist, r.iterations)
                    r.admitted = clock() - t0
                    running[(r.nbins, r.ticket)] = r
                except tgv.TgvError as e:
                    if e.status != 3:
                        raise
                    blocked.add(r.nbins)
                    keep.append(r)
            pending = keep
            max_running = max(max_running, len(running))
            # one round of iterations on every busy server
            finished_now = []
            events = []
            for n, srv in self.servers.items():
                if srv.running == 0:
                    continue
                srv.step(self.round_iters)
                ev = torch.cuda.Event()
                ev.record(self.streams[n])
                events.append(ev)
            for key in running:
                if key not in finishing and self.servers[key[0]].done(key[1]):
                    finished_now.append(key)
                    finishing.add(key)
            # finish the previous round on the host while this one runs
            for ev in in_flight_events(in_flight):
                ev.synchronize()
            for key in flush(in_flight):
                finishing.discard(key)
                r = running.pop(key)
                u = self.servers[key[0]].extract(key[1])
                r.finished = clock() - t0
                r.hist = None
                if self.keep:
                    r.u = u
                done += 1
            in_flight = [(events, finished_now)]
            rounds += 1
            if not running and not pending and not finished_now and nxt < len(reqs):
                time.sleep(max(0.0, reqs[nxt].arrival - (clock() - t0)))
        lat = np.array([r.finished - r.arrival for r in reqs])
        wait = np.array([r.admitted - r.arrival for r in reqs])
        vu = sum(srv.voxel_updates for srv in self.servers.values()) - vu0
        return StreamResult(lat, wait, clock() - t0, vu, done, max_running, rounds, reqs if self.keep else [])


def in_flight_events(in_flight):
    for events, _ in in_flight:
        yield from events


def flush(in_flight):
    for _, keys in in_flight:
        yield from keys


@dataclass
class PartChunk:
    """One treetop part of a level as an independent problem (its bricks active, its border
    frozen): DomainDesc-like fields plus the part's brick indices in the level."""
    origin: np.ndarray
    h: float
    bricks: np.ndarray
    frozen: Optional[np.ndarray]
    frozen_u: Optional[np.ndarray]
    frozen_v: Optional[np.ndarray]
    level_bricks: np.ndarray  # indices of the part's bricks in the level's brick list
    radius: float = 0.0

    @property
    def nbricks(self) -> int:
        return int(self.bricks.shape[0])

    @property
    def nvox(self) -> int:
        return 512 * self.nbricks


def part_chunks(level, brick_part: np.ndarray, u: np.ndarray, v: Optional[np.ndarray] = None) -> List[PartChunk]:
    """Chunks of a level's treetop parts (Sec. 4.3: parts are solved independently; Sec.
    4.5: the cubes of a part form the set A, its neighbouring cubes the set B whose
    indicator stays fixed).  Part k's bricks (brick_part == k, parts numbered 0..K-1)
    are active; every other brick of the level among their 26 neighbours is frozen with
    its values from `u` (per voxel, the level's brick order, 512 per brick) and `v`
    ((voxels, 3); zero if None) -- for a coarse-to-fine solve, the level's state after
    tgv_prolong, i.e. the parent level's indicator.  Bricks of other levels or outside
    the level are not part of the border (no link there)."""
    b = np.asarray(level.bricks, np.int32).reshape(-1, 3)
    index = {tuple(x): i for i, x in enumerate(b.tolist())}
    u = np.asarray(u, np.float32).reshape(-1, 512)
    v = np.zeros((b.shape[0] * 512, 3), np.float32) if v is None else np.asarray(v, np.float32).reshape(-1, 3)
    vb = v.reshape(-1, 512, 3).transpose(0, 2, 1)  # [brick][component][512]
    offs = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1) if (dx, dy, dz) != (0, 0, 0)]
    out = []
    for k in range(int(brick_part.max()) + 1):
        mine = np.nonzero(brick_part == k)[0]
        if len(mine) == 0:
            continue
        own = set(mine.tolist())
        ring = set()
        for i in mine.tolist():
            x, y, z = b[i]
            for dx, dy, dz in offs:
                j = index.get((x + dx, y + dy, z + dz))
                if j is not None and j not in own:
                    ring.add(j)
        ring = np.array(sorted(ring), np.int64)
        out.append(PartChunk(np.asarray(level.origin, np.float64), float(level.h), b[mine],
                             b[ring] if len(ring) else None, u[ring] if len(ring) else None,
                             vb[ring] if len(ring) else None, mine, float(getattr(level, "radius", 0.0) or 0.0)))
    return out


def batch_domain(U: UnionLevel, nbins: int, storage: str, stream: int, choice: dict) -> "tgv.Domain":
    """A domain over union level U set up for an autotuner choice (autotune.tune_batch)."""
    x = choice["run_length"] if choice["form"] == "union_graph" else 0
    return tgv.Domain([U], nbins=nbins, storage=storage, stream=stream, iter_kernel=choice["iter_kernel"], x_run=x)


def run_batch(dom: "tgv.Domain", U: UnionLevel, iterations: int, choice: dict):
    """`iterations` iterations of every chunk of U in the chosen form: the union level's
    launches replayed as a CUDA graph, or one persistent launch (tgv_solve_chunks)."""
    if choice["form"] == "union_graph":
        dom.solve_graph(0, iterations)
    else:
        dom.solve_chunks(0, U.first, [iterations] * len(U.ranges), run_length=choice["run_length"])


# Chunks per union level.  One union over a whole mix is slower than several smaller ones
# solved one after another: the fused kernel's rate falls with the size of the level it
# sweeps (dense 256^3 33.0 G voxel-updates/s, 352^3 29.9 G, 448^3 28.9 G; the 256-chunk
# c4 mix as one union 26.4 G, as unions of 32 chunks 29.4 G, of 8 chunks 30.7 G (FP32);
# holding 40 GB of other device memory changes nothing).  Groups of about 12 M active
# voxels still give every CTA of the grid many work items.
GROUP_VOXELS = 12 << 20


def group_chunks(sizes: Sequence[int], max_voxels: int = GROUP_VOXELS) -> List[List[int]]:
    """Consecutive chunks packed into groups of at most `max_voxels` active voxels (a chunk
    larger than that forms a group alone); max_voxels <= 0: one group of every chunk."""
    if max_voxels <= 0:
        return [list(range(len(sizes)))] if len(sizes) else []
    groups, cur, tot = [], [], 0
    for k, n in enumerate(sizes):
        if cur and tot + int(n) > max_voxels:
            groups.append(cur)
            cur, tot = [], 0
        cur.append(k)
        tot += int(n)
    if cur:
        groups.append(cur)
    return groups


class BatchGroups:
    """A chunk mix solved as union levels of grouped chunks (group_chunks), one domain per
    group, each set up for an autotuner choice (autotune.tune_batch; its "group_voxels"
    sets the group size, GROUP_VOXELS when absent).  `hists[k]`: chunk k's counts (torch
    tensors or numpy arrays, one row per active voxel)."""

    def __init__(self, chunks: Sequence, hists: Sequence, nbins: int, storage: str, stream: int, choice: dict,
                 max_voxels: Optional[int] = None):
        mv = choice.get("group_voxels", GROUP_VOXELS) if max_voxels is None else max_voxels
        self.choice = choice
        self.groups = group_chunks([c.nvox for c in chunks], mv)
        self.levels = [union_level([chunks[k] for k in g]) for g in self.groups]
        self.domains = []
        try:
            for g, U in zip(self.groups, self.levels):
                d = batch_domain(U, nbins, storage, stream, choice)
                self.domains.append(d)
                hs = [hists[k] for k in g]
                if hasattr(hs[0], "cpu"):
                    import torch
                    d.set_histograms(0, torch.cat(hs))
                else:
                    d.set_histograms(0, np.concatenate([np.asarray(h) for h in hs]))
        except Exception:
            self.close()
            raise

    def run(self, iterations: int):
        """`iterations` iterations of every chunk, group after group (asynchronous)."""
        for d, U in zip(self.domains, self.levels):
            run_batch(d, U, iterations, self.choice)

    def reset(self):
        for d in self.domains:
            d.reset(0)

    def field(self, chunk: int, name: str) -> np.ndarray:
        """Field `name` of chunk `chunk` (index into the chunks given), its active bricks only."""
        for g, U, d in zip(self.groups, self.levels, self.domains):
            if chunk in g:
                a, b = U.ranges[g.index(chunk)]
                return d.field(0, name)[a * 512:b * 512]
        raise IndexError(chunk)

    @property
    def launches(self) -> int:
        return sum(d.launches for d in self.domains)

    def close(self):
        for d in self.domains:
            d.close()
        self.domains = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
