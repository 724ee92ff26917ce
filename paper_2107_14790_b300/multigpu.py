"""Sharding of independent work across ranks (one process per GPU).

The method's parts are independent problems: treetop-leaf parts with frozen
borders (Sec. 4.3, Sec. 4.5) and, in the benchmark, whole instances.  Ranks
therefore split the units and never exchange data on the solve path; the
only collectives are on the host side of a benchmark: the slowest rank's
time and the totals.
"""
from __future__ import annotations

import os
import socket
import subprocess
import sys
from typing import Dict, List, Optional, Sequence

import numpy as np


def shard(costs: Sequence[float], rank: int, world: int) -> List[int]:
    """Indices of the units rank `rank` of `world` owns.

    Greedy longest-processing-time assignment: units in decreasing cost (ties by
    index) go to the currently least loaded rank (ties to the lower rank), so
    every rank computes the same partition without communicating.
    """
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = np.zeros(world)
    owner = np.empty(len(costs), np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += float(costs[i])
    return [i for i in range(len(costs)) if owner[i] == rank]


def reduce_scalar(value: float, op: str = "max") -> float:
    """Reduces a host scalar over the default process group (returns it unchanged without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM, "min": dist.ReduceOp.MIN}[op])
    return float(t.item())


def free_port() -> int:
    """A free TCP port on 127.0.0.1 for a rendezvous."""
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def launched_as_rank() -> bool:
    """True inside a process started by torch.distributed.run (or with WORLD_SIZE set)."""
    return "WORLD_SIZE" in os.environ


def relaunch(nproc: int, script: str, argv: Sequence[str], port: Optional[int] = None,
             env: Optional[Dict[str, str]] = None) -> int:
    """Runs `script argv` as `nproc` ranks of one node under torch.distributed.run
    (rendezvous on 127.0.0.1) and returns the launcher's exit code.  Each rank reads
    RANK / LOCAL_RANK / WORLD_SIZE / MASTER_ADDR / MASTER_PORT from its environment."""
    if nproc < 1:
        raise ValueError("nproc must be >= 1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={int(nproc)}",
           "--master-addr=127.0.0.1", f"--master-port={int(port or free_port())}", script, *argv]
    return subprocess.run(cmd, env=dict(os.environ, **(env or {}))).returncode


def gather_dict(local: dict) -> dict:
    """Merges every rank's dict of results on every rank (host objects over the default
    process group; returns `local` unchanged without one)."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return dict(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, local)
    out = {}
    for p in parts:
        out.update(p)
    return out
