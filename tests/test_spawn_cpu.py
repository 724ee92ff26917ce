"""The N-rank launch path on CPU: `multigpu.relaunch` (what `bench.py --gpus N` calls when it
is not already a rank) starts N processes under torch.distributed.run on 127.0.0.1; with gloo
they shard independent chunks, and the gathered per-chunk results equal the one-rank run
bit for bit.  `bench.py --gpus 2` itself relaunches and prints one line from rank 0."""
import json
import os
import subprocess
import sys

import numpy as np

from paper_2107_14790_b300.multigpu import relaunch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPT = os.path.join(ROOT, "tests", "_rank_script.py")


def test_relaunch_two_ranks_equals_one(tmp_path):
    env = dict(CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    one, two = tmp_path / "one.npz", tmp_path / "two.npz"
    assert relaunch(1, SCRIPT, [str(one)], env=env) == 0
    assert relaunch(2, SCRIPT, [str(two)], env=env) == 0
    a, b = np.load(one), np.load(two)
    assert int(a["world"]) == 1 and int(b["world"]) == 2
    assert float(a["units"]) == float(b["units"])
    keys = sorted(k for k in a.files if k.startswith("chunk"))
    assert keys == sorted(k for k in b.files if k.startswith("chunk")) and len(keys) == 6
    for k in keys:
        np.testing.assert_array_equal(a[k], b[k])


def test_bench_gpus_2_relaunches_and_prints_one_line():
    out = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--impl", "reference", "--small", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
