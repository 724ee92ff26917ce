"""One rank of the sharded chunk solve, started by multigpu.relaunch (torch.distributed.run).

Reads its rank from the environment, takes its share of independent chunks (multigpu.shard),
solves them with the FP64 oracle standing in for the device solve, merges every rank's
results (multigpu.gather_dict over gloo) and, on rank 0, saves them to the path argv[1].
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch.distributed as dist  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2107_14790_b300.multigpu import gather_dict, reduce_scalar, shard  # noqa: E402


def main(out_path):
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = synth.chunk_workload(9, 6, 2 * 512, 14 * 512, (8, 8), (5, 5))
    mine = shard([sp.domain.nvox for sp in specs], rank, world)
    res = {}
    for k in mine:
        lvl = oracle.OracleLevel(specs[k].domain, 8)
        lvl.hist[:] = specs[k].hist
        lvl.iterate(specs[k].iterations, nthreads=1)
        res[k] = lvl.u
    merged = gather_dict(res)
    units = reduce_scalar(sum(specs[k].domain.nvox for k in mine), "sum")
    if rank == 0:
        np.savez(out_path, world=world, units=units, owners=np.array([len(mine)]),
                 **{f"chunk{k}": v for k, v in merged.items()})
    dist.destroy_process_group()


if __name__ == "__main__":
    main(sys.argv[1])
