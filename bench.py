#!/usr/bin/env python3
"""Benchmark of the histogram + TGV primal-dual hot path on one B300 (or N, weak scaling).

Workload (one "step" = the whole hot path over one batch of synthetic input):
  dense 256^3 terrain domain (32^3 bricks of 8^3 voxels), 64 depth maps 512x512,
  10 histogram bins, 500 primal-dual iterations, energy/gap every 25 iterations:
    reset -> depth pyramids + Alg. 1 histograms (64 maps) -> 20 x (25 fused
    iterations + energy/gap reduction).
Metric: voxel-updates/s = active voxels x iterations / step time.

Output: one JSON line (rank 0).  Under torchrun every rank solves its own
independent instance (different seed): weak scaling, no collective on the path.
`--impl reference` times the FP64 CPU oracle instead (bounded sample per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="dense-256^3-terrain-64x512^2-maps-10bins-500it", n=256, nmaps=64, res=512, nbins=10,
                iterations=500, check_every=25)
SMALL = dict(workload="dense-64^3-sphere-16x128^2-maps-8bins-200it", n=64, nmaps=16, res=128, nbins=8,
             iterations=200, check_every=25)
ITER_KERNEL_SRCS = [os.path.join(ROOT, "paper_2107_14790_b300", "csrc", f)
                    for f in ("tgv_solve.cu", "tgv_iter_pipe.cu", "tgv_iter_pair.cu", "tgv_internal.cuh", "tgv_async.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "tgv_iter_kernel_dense256_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--small", action="store_true", help="64^3 sphere case instead of the 256^3 terrain")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--iter-kernel", default="paired", choices=["paired", "pipelined", "one_brick_per_cta"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", type=int, default=0, metavar="N",
                    help="profiling case: N^3 dense domain, seeded random 10-bin histograms, "
                         "warm-up + 4 fused iterations + one energy/gap (no depth maps)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_scene(cfg, seed, device):
    import synth
    if cfg["n"] == 64:
        return synth.sphere_scene(seed=seed)
    return synth.terrain_scene(seed=seed, n=cfg["n"], nmaps=cfg["nmaps"], res=cfg["res"], nbins=cfg["nbins"],
                               iterations=cfg["iterations"], device=device)


def algorithmic_bytes_per_voxel(nbins: int, storage: str) -> int:
    """One fused iteration reads u, ubar, v, vbar, p, q, hist and writes u, ubar, v, vbar, p, q once."""
    s = 4 if storage == "fp32" else 2
    state = 4 + 4 + (3 + 3 + 3 + 6) * s
    return 2 * state + 2 * nbins


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in ITER_KERNEL_SRCS:
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------- ours
def run_ours(args, cfg):
    import torch
    import torch.distributed as tdist
    from paper_2107_14790_b300 import build, tgv

    rank, world, local = dist_env()
    if world > 1:
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    tgv.lib()
    stream = torch.cuda.Stream()
    seed = 1002 + 1000 * rank if cfg["n"] != 64 else 1001 + 1000 * rank
    sc = make_scene(cfg, seed, f"cuda:{local}")
    nbins = cfg["nbins"]
    depth_host = torch.from_numpy(np.stack(sc.depths).astype(np.float32)).pin_memory()
    with torch.cuda.stream(stream):
        depth_dev = depth_host.to(f"cuda:{local}", non_blocking=True)
    stream.synchronize()
    dom = tgv.Domain([sc.domain], nbins=nbins, storage=args.storage, stream=stream.cuda_stream,
                     iter_kernel=args.iter_kernel)
    nvox = dom.voxels(0)
    iters, ce = cfg["iterations"], cfg["check_every"]
    blocks = [ce] * (iters // ce) + ([iters % ce] if iters % ce else [])

    def step(ev=None, energies=None):
        dom.reset(0, clear_hist=True)
        dom.accumulate(0, sc.cameras, depth_dev)
        for k, nb in enumerate(blocks):
            if ev is not None:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            tgv.tgv_solve(dom.handle, 0, nb, False)
            if ev is not None:
                e1.record(stream)
                ev.append((e0, e1, nb))
            e = dom.energy(0)
            if energies is not None:
                energies.append(e)

    def barrier():
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 0)):
        step()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev_list, energies = [], []
    l0 = dom.launches
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(ev_list, energies)
    t1.record(stream)
    barrier()
    ck = clocks.stop()
    launches = dom.launches - l0
    ms = t0.elapsed_time(t1)
    if world > 1:
        tt = torch.tensor([ms], device=f"cuda:{local}")
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        ms = float(tt.item())
    ms_per_step = ms / args.steps
    value = world * nvox * iters * args.steps / (ms / 1e3)
    # dominant kernel: the fused iteration; mean launch duration from the events around its launches
    it_ms = sum(a.elapsed_time(b) for a, b, _ in ev_list)
    it_launches = sum(n for _, _, n in ev_list)
    per_launch_s = it_ms / 1e3 / it_launches
    bpv = algorithmic_bytes_per_voxel(nbins, args.storage)
    achieved = nvox * bpv / per_launch_s / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except Exception:
        peak, peak_src = 6400.0, "fallback"
    traffic = None
    try:
        tr = json.load(open(TRAFFIC_FILE))
        if (tr.get("kernel_sha") == kernel_hash() and tr.get("storage", "fp32") == args.storage
                and tr.get("iter_kernel") == args.iter_kernel):
            traffic = tr["dram_bytes_per_launch"]
    except Exception:
        pass
    last = energies[-1]
    result = {
        "metric": "TGV voxel-updates/s (histograms + 500 fused primal-dual iterations + energy/gap)",
        "value": value, "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.storage == "fp32" else f"f32-math/{args.storage}-storage",
        "data": "synthetic (seeded terrain scene, ray-cast depth maps)",
        "config": {"workload": cfg["workload"], "voxels": nvox, "maps": cfg["nmaps"], "map_res": cfg["res"],
                   "nbins": nbins, "iterations": iters, "energy_every": ce, "storage": args.storage,
                   "l2": "inputs larger than L2 (state %.2f GB)" % (dom.nbytes / 1e9),
                   "parallelism": f"independent instance per GPU x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": peak_src,
                     "kernel": {"paired": "tgv_iter_pair_kernel", "pipelined": "tgv_iter_pipe_kernel",
                                "one_brick_per_cta": "tgv_iter_kernel"}[args.iter_kernel],
                     "algorithmic_bytes_per_voxel": bpv, "mean_launch_us": per_launch_s * 1e6},
        "energy_gap": {"energy": last[0], "dual": last[1], "gap": last[2], "certified": bool(last[3])},
        "gpu_launches": launches,
        "clocks": ck,
    }
    # end to end through the public API with host buffers: H2D of the maps, D2H of u
    if not args.no_e2e:
        u_host = torch.empty((nvox, 1), dtype=torch.float32).pin_memory()
        barrier()
        e0 = time.perf_counter()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                depth_dev.copy_(depth_host, non_blocking=True)
            step()
            tgv.tgv_extract_field(dom.handle, 0, "u", u_host.numpy())
        barrier()
        e_s = time.perf_counter() - e0
        if world > 1:
            tt = torch.tensor([e_s], device=f"cuda:{local}")
            tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
            e_s = float(tt.item())
        result["e2e"] = {"value": world * nvox * iters * args.steps / e_s, "unit": "voxel-updates/s",
                         "h2d_bytes_per_step": int(depth_host.numel() * 4),
                         "d2h_bytes_per_step": int(nvox * 4 + 8 * 4 * len(blocks))}
    dom.close()
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(cfg, sc)
    if world > 1:
        tdist.destroy_process_group()
    return result if rank == 0 else None


# ------------------------------------------------------------------------------------------- oracle
def oracle_sample(cfg, sc, bricks_per_axis=8, iters=100):
    """Oracle on a bounded sample of the workload: a block of bricks at the domain centre,
    histograms from all maps, then `iters` TGV iterations.  Returns (updates/s, seconds, note)."""
    import oracle
    import synth
    nb = cfg["n"] // 8
    lo = max(0, nb // 2 - bricks_per_axis // 2)
    k = min(bricks_per_axis, nb)
    bricks = synth.dense_bricks(k, k, k, offset=(lo, lo, lo))
    desc = synth.DomainDesc(sc.domain.origin, sc.domain.h, bricks)
    lvl = oracle.OracleLevel(desc, cfg["nbins"])
    t0 = time.perf_counter()
    for cam, d in zip(sc.cameras, sc.depths):
        lvl.accumulate(cam, d, 1)
    lvl.iterate(iters)
    lvl.energy()
    dt = time.perf_counter() - t0
    return lvl.n * iters / dt, dt, f"{k}^3 bricks ({lvl.n} voxels) at the domain centre, all {len(sc.cameras)} maps, {iters} iterations + energy"


def cpu_baseline(cfg, sc):
    import oracle
    ups, dt, note = oracle_sample(cfg, sc)
    return {"value": ups, "unit": "voxel-updates/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": note, "seconds": dt}


def run_reference(args, cfg):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    import oracle
    dev = "cpu"
    try:
        import torch
        if torch.cuda.is_available():
            dev = f"cuda:{local}"  # scene generation only; the timed work is the CPU oracle
    except Exception:
        pass
    sc = make_scene(cfg, 1002 if cfg["n"] != 64 else 1001, dev)
    for _ in range(max(args.warmup, 0)):
        oracle_sample(cfg, sc, bricks_per_axis=4, iters=20)
    vals, secs = [], []
    note = ""
    for _ in range(args.steps):
        ups, dt, note = oracle_sample(cfg, sc)
        vals.append(ups)
        secs.append(dt)
    value = statistics.median(vals)
    cores = oracle.max_threads()
    return {"impl": "reference", "metric": "TGV voxel-updates/s (histograms + 500 fused primal-dual iterations + energy/gap)",
            "value": value, "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(secs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded terrain scene, ray-cast depth maps)",
            "config": {"workload": cfg["workload"], "sample": note},
            "cpu_baseline": {"value": value, "unit": "voxel-updates/s", "cores": cores, "kind": "oracle",
                             "sample": note},
            "e2e": {"value": value, "unit": "voxel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_case(args):
    """A small case of the same kernels for ncu: larger than L2, a few hundred MB on the device."""
    import torch
    import synth
    from paper_2107_14790_b300 import build, tgv
    build.build()
    n = args.profile
    desc = synth.DomainDesc(np.zeros(3), 1.0 / n, synth.dense_bricks(n // 8))
    hist = synth.random_histograms(np.random.default_rng(7), desc.nvox, 10, max_count=20)
    stream = torch.cuda.Stream()
    dom = tgv.Domain([desc], nbins=10, storage=args.storage, stream=stream.cuda_stream,
                     iter_kernel=args.iter_kernel)
    dom.set_histograms(0, hist)
    tgv.tgv_solve(dom.handle, 0, 6, False)
    tgv.tgv_solve(dom.handle, 0, 4, False)
    e = dom.energy(0)
    dom.close()
    print(json.dumps({"profile_case": n, "voxels": desc.nvox, "energy": list(map(float, e))}))


def main():
    args = parse()
    if args.profile:
        run_profile_case(args)
        return
    cfg = SMALL if args.small else WORKLOAD
    if args.impl == "reference":
        res = run_reference(args, cfg)
    else:
        res = run_ours(args, cfg)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
