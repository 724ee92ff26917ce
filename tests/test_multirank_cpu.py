"""The multi-rank path on CPU: two gloo ranks shard independent chunks, solve their own
share (with the FP64 oracle standing in for the device solve), and the gathered results
equal a single-rank run; the benchmark's timing reduction takes the slowest rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2107_14790_b300.multigpu import shard


def test_shard_partitions_and_balances():
    costs = [5, 1, 9, 3, 3, 7, 2, 8]
    parts = [shard(costs, r, 3) for r in range(3)]
    allidx = sorted(i for p in parts for i in p)
    assert allidx == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    assert parts == [shard(costs, r, 3) for r in range(3)]  # deterministic
    with pytest.raises(ValueError):
        shard(costs, 3, 3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    import oracle
    import synth
    from paper_2107_14790_b300.multigpu import reduce_scalar, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = synth.chunk_workload(7, 5, 2 * 512, 12 * 512, (8, 8), (6, 6))
    mine = shard([sp.domain.nvox * sp.iterations for sp in specs], rank, world)
    res = {}
    for k in mine:
        lvl = oracle.OracleLevel(specs[k].domain, 8)
        lvl.hist[:] = specs[k].hist
        lvl.iterate(specs[k].iterations, nthreads=1)
        res[k] = lvl.u
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    t_max = reduce_scalar(1.0 + rank, "max")
    units = reduce_scalar(sum(specs[k].domain.nvox * specs[k].iterations for k in mine), "sum")
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        np.savez(os.path.join(out_dir, "ranks.npz"), t_max=t_max, units=units,
                 **{f"u{k}": v for k, v in merged.items()})
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one(tmp_path):
    import oracle
    import synth
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = np.load(tmp_path / "ranks.npz")
    specs = synth.chunk_workload(7, 5, 2 * 512, 12 * 512, (8, 8), (6, 6))
    assert float(got["t_max"]) == 2.0
    assert float(got["units"]) == sum(sp.domain.nvox * sp.iterations for sp in specs)
    for k, sp in enumerate(specs):
        lvl = oracle.OracleLevel(sp.domain, 8)
        lvl.hist[:] = sp.hist
        lvl.iterate(sp.iterations)
        np.testing.assert_array_equal(got[f"u{k}"], lvl.u)
