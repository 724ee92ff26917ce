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
# sources that define each form of the fused iteration kernel (the traffic counters are
# valid only for the sources they were taken on)
ITER_KERNEL_SRCS = {form: [os.path.join(ROOT, "paper_2107_14790_b300", "csrc", f)
                           for f in (main, "tgv_internal.cuh", "tgv_async.cuh", "tgv_pair_cta.cuh")]
                    for form, main in (("paired", "tgv_iter_pair.cu"), ("pipelined", "tgv_iter_pipe.cu"),
                                       ("one_brick_per_cta", "tgv_solve.cu"))}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "tgv_iter_kernel_dense256_traffic.json")
TRAFFIC_FILE_FX16 = os.path.join(ROOT, "profiles", "tgv_iter_kernel_dense256_traffic_fx16.json")


def measured_traffic(path, storage, nvox, nbins, form="paired"):
    """DRAM bytes per launch of the fused kernel from a committed 1-pass ncu capture, or None
    when the capture does not match (other sources, storage, size or bins)."""
    try:
        tr = json.load(open(path))
        if (tr.get("kernel_sha") == kernel_hash(form) and tr.get("storage", "fp32") == storage
                and tr.get("voxels", 16777216) == nvox and tr.get("nbins", 10) == nbins
                and tr.get("iter_kernel") == form):
            return tr["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--small", action="store_true", help="64^3 sphere case instead of the 256^3 terrain")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16", "fx16"])
    ap.add_argument("--iter-kernel", default="paired", choices=["paired", "pipelined", "one_brick_per_cta"])
    ap.add_argument("--x-run", type=int, default=0, help="paired kernel: work items per run (0 = automatic)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched block of the default line")
    ap.add_argument("--no-reduced", action="store_true", help="skip the 16-bit storage block of the default line")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving block of the default line")
    ap.add_argument("--block-chunks", type=int, default=32, help="batched block: chunks (c4's size distribution)")
    ap.add_argument("--block-requests", type=int, default=200, help="serving block: requests")
    ap.add_argument("--group-voxels", type=int, default=None,
                    help="batched forms: active voxels per union of grouped chunks (default: the tuned choice)")
    ap.add_argument("--workload", default="dense", choices=["dense", "batched", "serving", "multilevel", "lidar", "mesh", "octree", "composite",
                             "histforms", "precision"],
                    help="dense: the 256^3 terrain (default line); batched: 256 chunks 32^3..192^3, "
                         "300 iterations; serving: Poisson stream of 2000 chunk-solve requests")
    ap.add_argument("--requests", type=int, default=2000, help="serving: number of requests")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serving: HBM budget of all arenas")
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


def state_bytes(nvox: int, nbins: int, storage: str) -> int:
    """Device bytes of a level's iteration state and histograms (what both arms print as the
    working set): u, ubar x2, v, vbar x2, p x2, q x2 and the packed 16-bit counts."""
    s = 4 if storage == "fp32" else 2
    return nvox * (4 + 2 * 4 + (3 + 2 * 3 + 2 * 3 + 2 * 6) * s + 4 * ((nbins + 1) // 2))


def kernel_hash(form: str = "paired") -> str:
    h = hashlib.sha256()
    for p in ITER_KERNEL_SRCS[form]:
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
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
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
                     iter_kernel=args.iter_kernel, x_run=args.x_run)
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
    traffic = measured_traffic(TRAFFIC_FILE if args.storage == "fp32" else TRAFFIC_FILE_FX16, args.storage, nvox, nbins,
                               args.iter_kernel)
    last = energies[-1]
    result = {
        "metric": "TGV voxel-updates/s (histograms + %d fused primal-dual iterations + energy/gap)" % iters,
        "value": value, "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.storage == "fp32" else f"f32-math/{args.storage}-storage",
        "data": scene_note(cfg),
        "config": arm_config(cfg, args, nvox, world),
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
    u_ref = dom.field(0, "u")[:, 0].copy()
    dom.close()
    if not args.no_reduced and not args.small and args.storage == "fp32":
        rb = reduced_block(sc, cfg, depth_dev, stream, u_ref)
        rb["frac"] = rb["achieved_gbs"] / peak
        rb["traffic"] = measured_traffic(TRAFFIC_FILE_FX16, "fx16", nvox, nbins)
        rb["speedup_over_fp32"] = rb["voxel_updates_per_s"] / value
        result["reduced_precision"] = rb
    del depth_dev
    torch.cuda.empty_cache()
    # bounded blocks of the batched and served forms (the metric's chunk-solve latency)
    if not args.no_batched and not args.small:
        result["batched"] = batched_block(stream, rank, world, local, nchunks=args.block_chunks,
                                          group_voxels=args.group_voxels)
    if not args.no_serving and not args.small:
        from paper_2107_14790_b300.multigpu import gather_dict, reduce_scalar
        sv = serving_block("fp32", args.block_requests, 60.0, rank=rank)
        lat = np.concatenate(list(gather_dict({rank: sv.pop("latencies")}).values()))
        span = reduce_scalar(sv["makespan_s"], "max")
        vu = reduce_scalar(sv["voxel_updates_per_s"] * sv["makespan_s"], "sum")
        sv["latency_s"] = {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())}
        sv["voxel_updates_per_s"] = vu / span
        sv["ranks"] = world
        result["serving"] = sv
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


def scene_note(cfg):
    kind = "sphere" if cfg["n"] == 64 else "terrain"
    return f"synthetic (seeded {kind} scene, ray-cast depth maps)"


def arm_config(cfg, args, nvox, world):
    """The workload description both arms print (identical for the same arguments)."""
    nbytes = state_bytes(nvox, cfg["nbins"], args.storage)
    return {"workload": cfg["workload"], "voxels": nvox, "maps": cfg["nmaps"], "map_res": cfg["res"],
            "nbins": cfg["nbins"], "iterations": cfg["iterations"], "energy_every": cfg["check_every"],
            "storage": args.storage,
            "l2": ("inputs larger than L2 (state %.2f GB)" if nbytes > 126e6 else
                   "state fits in L2 (%.2f GB): a parity case, not a roofline case") % (nbytes / 1e9),
            "parallelism": f"independent instance per GPU x{world}"}


def oracle_full_sphere():
    """The whole 64^3 sphere workload (16 maps 128^2, 8 bins, 200 iterations + energy) on the
    oracle: the one configuration the oracle finishes in full within seconds."""
    import oracle
    import synth
    sc = synth.sphere_scene()
    lvl = oracle.OracleLevel(sc.domain, sc.nbins)
    t0 = time.perf_counter()
    for cam, d in zip(sc.cameras, sc.depths):
        lvl.accumulate(cam, d, 1)
    lvl.iterate(SMALL["iterations"])
    lvl.energy()
    dt = time.perf_counter() - t0
    return {"workload": SMALL["workload"], "value": lvl.n * SMALL["iterations"] / dt, "unit": "voxel-updates/s",
            "seconds": dt}


def cpu_baseline(cfg, sc):
    import oracle
    ups, dt, note = oracle_sample(cfg, sc)
    out = {"value": ups, "unit": "voxel-updates/s", "cores": oracle.max_threads(), "kind": "oracle",
           "sample": note, "seconds": dt}
    if cfg["n"] != 64:
        upd = sc.domain.nvox * cfg["iterations"]
        out["why_a_sample"] = ("the full workload is %.2g voxel-updates, about %.0f minutes of the oracle at this "
                               "rate: beyond the few-minute bound of a benchmark run" % (upd, upd / ups / 60))
        out["full_sphere_64"] = oracle_full_sphere()
    return out


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
    return {"impl": "reference", "metric": "TGV voxel-updates/s (histograms + %d fused primal-dual iterations + energy/gap)" % cfg["iterations"],
            "value": value, "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(secs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": scene_note(cfg),
            "config": arm_config(cfg, args, sc.domain.nvox, world),
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
                     iter_kernel=args.iter_kernel, x_run=args.x_run)
    dom.set_histograms(0, hist)
    tgv.tgv_solve(dom.handle, 0, 6, False)
    tgv.tgv_solve(dom.handle, 0, 4, False)
    e = dom.energy(0)
    dom.close()
    print(json.dumps({"profile_case": n, "voxels": desc.nvox, "energy": list(map(float, e))}))


def reduced_block(sc, cfg, depth_dev, stream, u_ref, storage="fx16", steps=3):
    """The default workload with 16-bit storage of v, vbar, p, q: the same step (reset,
    histograms, the configured iterations with energy/gap checks), timed over `steps` steps;
    the fused kernel's mean launch time and its algorithmic bandwidth; max and RMS of the
    final u against the FP32 run's (the stated accuracy of the reduced forms: 5e-3)."""
    import torch
    from paper_2107_14790_b300 import tgv
    nbins, iters, ce = cfg["nbins"], cfg["iterations"], cfg["check_every"]
    blocks = [ce] * (iters // ce) + ([iters % ce] if iters % ce else [])
    dom = tgv.Domain([sc.domain], nbins=nbins, storage=storage, stream=stream.cuda_stream)
    nvox = dom.voxels(0)

    def step(ev=None):
        dom.reset(0, clear_hist=True)
        dom.accumulate(0, sc.cameras, depth_dev)
        for nb in blocks:
            if ev is not None:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            tgv.tgv_solve(dom.handle, 0, nb, False)
            if ev is not None:
                e1.record(stream)
                ev.append((e0, e1, nb))
            dom.energy(0)
    step()
    torch.cuda.synchronize()
    ev = []
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        step(ev)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    per_launch = sum(a.elapsed_time(b) for a, b, _ in ev) / sum(n for _, _, n in ev) / 1e3
    u = dom.field(0, "u")[:, 0]
    dom.close()
    d = np.abs(u.astype(np.float64) - u_ref.astype(np.float64))
    bpv = algorithmic_bytes_per_voxel(nbins, storage)
    return {"storage": storage, "voxel_updates_per_s": nvox * iters / (ms / 1e3), "ms_per_step": ms,
            "mean_launch_us": per_launch * 1e6, "algorithmic_bytes_per_voxel": bpv,
            "achieved_gbs": nvox * bpv / per_launch / 1e9, "u_err_inf_vs_fp32": float(d.max()),
            "u_err_rms_vs_fp32": float(np.sqrt(np.mean(d * d))), "steps": steps}


def batched_block(stream, rank, world, local, nchunks=32, iters=300, storages=("fp32", "fx16"), run_lengths=(16,),
                  tune=True, group_voxels=None):
    """Bounded form of the batched workload for the default line: `nchunks` chunks of the
    c4 size distribution (log-uniform 32^3..192^3 active voxels, frozen one-brick shell,
    10 bins, `iters` iterations), sharded over the ranks (strong scaling: each rank solves
    its own chunks, no collective on the path).  Forms per storage type: the persistent
    launch (tgv_solve_chunks: one kernel drains every chunk's runs behind per-chunk
    barriers, replayed as a CUDA graph), one union level with one launch per iteration
    replayed as a CUDA graph, the autotuner's choice over union levels of grouped chunks
    (batching.BatchGroups, about 12 M voxels per group, group after group); and the plain
    form (every chunk its own domain, FP32)."""
    import torch
    import synth
    from paper_2107_14790_b300 import tgv
    from paper_2107_14790_b300.batching import union_level
    from paper_2107_14790_b300.multigpu import reduce_scalar, shard
    geo = synth.chunk_workload(1004, nchunks, 32 ** 3, 192 ** 3, (10, 10), (iters, iters), hist="none")
    mine = shard([g.domain.nvox for g in geo], rank, world)
    specs = [geo[k] for k in mine]
    for sp in specs:
        sp.hist = synth.chunk_histogram(sp, f"cuda:{local}")
    nvox = sum(sp.domain.nvox for sp in specs)
    tot = reduce_scalar(nvox, "sum")
    U = union_level([sp.domain for sp in specs])
    hist = torch.cat([sp.hist for sp in specs])

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return reduce_scalar(e0.elapsed_time(e1), "max")

    out = {"chunks": nchunks, "voxels": int(tot), "iterations": iters, "l2": "inputs larger than L2 "
           "(state %.2f GB)" % (state_bytes(int(tot), 10, "fp32") / 1e9)}
    launches = 0
    first = U.first
    its = [iters] * len(specs)
    for storage in storages:
        dom = tgv.Domain([U], nbins=10, storage=storage, stream=stream.cuda_stream)
        dom.set_histograms(0, hist)
        dom.solve_graph(0, iters)  # first call: plain launches, captures the graph
        dom.reset(0)
        l0 = dom.launches
        ms = timed(lambda: dom.solve_graph(0, iters))
        launches += dom.launches - l0
        out[f"union_graph_{storage}"] = {"voxel_updates_per_s": tot * iters / (ms / 1e3), "ms": ms}
        for R in run_lengths:
            dom.reset(0)
            dom.solve_chunks(0, first, its, run_length=R)  # first call captures the graph
            dom.reset(0)
            l0 = dom.launches
            ms = timed(lambda: dom.solve_chunks(0, first, its, run_length=R))
            launches += dom.launches - l0
            key = f"persistent_{storage}" + ("" if len(run_lengths) == 1 else f"_R{R}")
            out[key] = {"voxel_updates_per_s": tot * iters / (ms / 1e3), "ms": ms, "run_length": R,
                        "launches": dom.launches - l0}
        dom.close()
    if tune:
        # the autotuner's choice for this chunk mix (timed on a sample of it, cached per mix)
        from paper_2107_14790_b300 import autotune
        from paper_2107_14790_b300.batching import BatchGroups
        for storage in storages:
            ch = autotune.tune_batch([sp.domain for sp in specs], 10, storage, hist_of=lambda dm, m={
                id(sp.domain): sp.hist for sp in specs}: m[id(dm)])
            # the chosen form over union levels of grouped chunks, group after group
            with BatchGroups([sp.domain for sp in specs], [sp.hist for sp in specs], 10, storage,
                             stream.cuda_stream, ch, max_voxels=group_voxels) as G:
                G.run(iters)
                G.reset()
                l0 = G.launches
                ms = timed(lambda: G.run(iters))
                launches += G.launches - l0
                out[f"autotuned_{storage}"] = {
                    "voxel_updates_per_s": tot * iters / (ms / 1e3), "ms": ms, "groups": len(G.groups),
                    "choice": {k: ch.get(k) for k in ("form", "iter_kernel", "run_length", "group_voxels")}}
                if group_voxels is not None:
                    out[f"autotuned_{storage}"]["choice"]["group_voxels"] = group_voxels
    doms = []
    for sp in specs:
        d = tgv.Domain([sp.domain], nbins=10, stream=stream.cuda_stream)
        d.set_histograms(0, sp.hist)
        doms.append(d)
    l0 = sum(d.launches for d in doms)
    ms = timed(lambda: [tgv.tgv_solve(d.handle, 0, iters, False) for d in doms])
    launches += sum(d.launches for d in doms) - l0
    out["plain_fp32"] = {"voxel_updates_per_s": tot * iters / (ms / 1e3), "ms": ms}
    for d in doms:
        d.close()
    base = out["plain_fp32"]["voxel_updates_per_s"]
    for key, rec in out.items():
        if isinstance(rec, dict) and key != "plain_fp32" and "voxel_updates_per_s" in rec:
            rec["speedup_over_plain_fp32"] = rec["voxel_updates_per_s"] / base
    out["gpu_launches"] = int(reduce_scalar(launches, "sum"))
    return out


def serving_block(storage, nreq, budget_gb, seed=1005, rank=0, overload=0):
    """Poisson stream of `nreq` chunk-solve requests (16k..8M active voxels, 8..12 bins,
    200..600 iterations) through one server per bin count: a saturation run (requests all
    arriving at once) gives the saturated rate; the stream then arrives at 0.8x that rate.
    `overload` > 0 adds a run of that many requests arriving at 2x the saturated rate.
    Returns p50/p99 latency, queue wait and voxel-updates/s (each rank its own requests)."""
    import torch
    import synth
    from paper_2107_14790_b300 import tgv
    from paper_2107_14790_b300.batching import Request, RequestStream
    specs = synth.chunk_workload(seed + 1000 * rank, nreq, 16 * 1024, 8 * 1024 * 1024, (8, 12), (200, 600),
                                 rate=1.0, hist="none")
    bins = sorted({sp.nbins for sp in specs})
    budget = budget_gb * 1e9
    streams = {n: torch.cuda.Stream() for n in bins}

    def brick_bytes(n):
        npairs = (n + 1) // 2
        sb = 4 if storage == "fp32" else 2
        return 512 * (4 + 8 + (3 + 6 + 6 + 12) * sb + 4 * npairs) + 48, 512 * (4 + 8 + 9 * sb)

    servers = {}
    for n in bins:
        ba, bf = brick_bytes(n)
        cap = int(budget / len(bins) / (ba + bf))
        servers[n] = tgv.Server(cap, cap, nbins=n, storage=storage, stream=streams[n].cuda_stream,
                                staging_bytes=64 << 20)

    def req(k, t):
        sp = specs[k]
        return Request(k, sp.domain, sp.nbins, sp.iterations, t, lambda sp=sp: synth.chunk_histogram(sp, "cuda"))

    RequestStream(servers, streams).run([req(k, 0.0) for k in range(min(8, nreq))])  # warm-up
    nsat = max(1, nreq // 2)
    sat = RequestStream(servers, streams).run([req(k, 0.0) for k in range(nsat)])
    sat_rate = nsat / sat.makespan
    rate = 0.8 * sat_rate
    main = RequestStream(servers, streams).run([req(k, specs[k].arrival / rate) for k in range(nreq)])
    p = lambda a, q: float(np.percentile(a, q))
    over = None
    if overload:
        o = RequestStream(servers, streams).run([req(k, specs[k].arrival / (2.0 * sat_rate))
                                                 for k in range(min(nreq, overload))])
        over = {"requests": o.completed, "p50": p(o.latencies, 50), "p99": p(o.latencies, 99),
                "voxel_updates_per_s": o.voxel_updates / o.makespan}
    for s_ in servers.values():
        s_.close()
    return {"requests": nreq, "budget_gb": budget_gb, "servers": len(servers), "storage": storage,
            "arrival_rate_per_s": rate, "saturated_rate_per_s": sat_rate,
            "latency_s": {"p50": p(main.latencies, 50), "p99": p(main.latencies, 99),
                          "mean": float(main.latencies.mean()), "max": float(main.latencies.max())},
            "queue_wait_s": {"p50": p(main.wait, 50), "p99": p(main.wait, 99)},
            "voxel_updates_per_s": main.voxel_updates / main.makespan, "makespan_s": main.makespan,
            "saturated_voxel_updates_per_s": sat.voxel_updates / sat.makespan, "max_running": main.max_running,
            "overload_2x": over, "latencies": main.latencies}


def run_batched(args):
    """256 uneven chunks (32^3..192^3 active voxels, frozen one-brick shell, 10 bins, 300
    iterations), sharded over the ranks: per storage form (FP32, FX16, FP16, BF16) the
    persistent launch, the union level's graph-replayed launches and the autotuner's choice,
    against the plain form (each chunk its own domain, FP32); and every form's accuracy on
    the 3 smallest chunks against the FP64 oracle (timed: the CPU baseline)."""
    import torch
    import torch.distributed as tdist
    import oracle
    import synth
    from paper_2107_14790_b300 import build, tgv
    from paper_2107_14790_b300.batching import union_level
    from paper_2107_14790_b300.multigpu import shard
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    build.build()
    iters, nchunks = 300, 256
    stream = torch.cuda.Stream()
    storages = ("fp32", "fx16", "fp16", "bf16")
    t0 = time.perf_counter()
    blk = batched_block(stream, rank, world, local, nchunks=nchunks, iters=iters, storages=storages,
                        group_voxels=args.group_voxels)
    t_blk = time.perf_counter() - t0
    # accuracy on this rank's 3 smallest chunks: each form against the FP64 oracle
    geo = synth.chunk_workload(1004, nchunks, 32 ** 3, 192 ** 3, (10, 10), (iters, iters), hist="none")
    mine = shard([g.domain.nvox for g in geo], rank, world)
    small = sorted(mine, key=lambda k: geo[k].domain.nbricks)[:3]
    specs = [geo[k] for k in small]
    for sp in specs:
        sp.hist = synth.chunk_histogram(sp, f"cuda:{local}")
    U = union_level([sp.domain for sp in specs])
    hist = torch.cat([sp.hist for sp in specs])
    t_cpu = time.perf_counter()
    ref = []
    for sp in specs:
        lvl = oracle.OracleLevel(sp.domain, sp.nbins)
        lvl.hist[:] = sp.hist.cpu().numpy()
        lvl.iterate(iters)
        ref.append(lvl.u)
    t_cpu = time.perf_counter() - t_cpu
    acc = {}
    for storage in storages:
        with tgv.Domain([U], nbins=10, storage=storage, stream=stream.cuda_stream) as dom:
            dom.set_histograms(0, hist)
            dom.solve_chunks(0, U.first, [iters] * len(specs))
            u = dom.field(0, "u")[:, 0]
        acc[storage] = max(float(np.max(np.abs(u[512 * a:512 * b] - r))) for (a, b), r in zip(U.ranges, ref))
    if world > 1:
        tdist.destroy_process_group()
    if rank != 0:
        return None
    best = max((v["voxel_updates_per_s"], k) for k, v in blk.items() if isinstance(v, dict) and "speedup_over_plain_fp32" in v)
    return {"metric": "batched chunk solve: voxel-updates/s (256 chunks 32^3..192^3, 300 iterations)",
            "value": best[0], "unit": "voxel-updates/s", "n_gpus": world,
            "scaling": "weak" if world == 1 else "strong", "higher_is_better": True,
            "dtype": "f32-math/%s-storage" % best[1].split("_")[-1], "data": "synthetic (seeded chunk scenes)",
            "config": {"workload": "batched-256-chunks-32^3..192^3-10bins-300it", "chunks": nchunks,
                       "voxels": blk["voxels"], "seconds": t_blk},
            "best_form": best[1], "batched": blk,
            "u_err_inf_vs_fp64_oracle": acc,
            "cpu_baseline": {"value": sum(sp.domain.nvox for sp in specs) * iters / t_cpu, "unit": "voxel-updates/s",
                             "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"the 3 smallest chunks, {iters} iterations each"},
            "accuracy_sample": f"3 smallest chunks vs FP64 oracle after {iters} iterations (persistent launch)"}


def run_multilevel(args):
    """Sparse three-level domain (~49M active voxels: terrain at level 0, a blob at 4x finer
    level 2, a level-1 transition shell), 256 maps 1024x1024, 10 bins, 200 iterations per
    level, coarse-to-fine with prolongation; FP32 and 16-bit storage of v, vbar, p, q."""
    import torch
    import synth
    from paper_2107_14790_b300 import build, tgv
    build.build()
    torch.cuda.set_device(0)
    t_gen = time.perf_counter()
    sc = synth.multilevel_scene(device="cuda")
    t_gen = time.perf_counter() - t_gen
    L, nb, iters = sc["levels"], sc["nbins"], sc["iterations"]
    depth = torch.from_numpy(np.stack(sc["depths"])).cuda()
    stream = torch.cuda.Stream()
    runs = {}
    for storage in ("fp32", "fp16", "bf16"):
        dom = tgv.Domain(L, nbins=nb, storage=storage, stream=stream.cuda_stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        ev[0].record(stream)
        for l in range(3):
            dom.accumulate(l, sc["cameras"], depth)
        ev[1].record(stream)
        dom.solve(0, iters)
        ev[2].record(stream)
        dom.prolong(0)
        ev[3].record(stream)
        dom.solve(1, iters)
        ev[4].record(stream)
        dom.prolong(1)
        ev[5].record(stream)
        dom.solve(2, iters)
        ev[6].record(stream)
        e = dom.energy(2)
        dom.synchronize()
        solve_ms = [ev[1 + 2 * k].elapsed_time(ev[2 + 2 * k]) for k in range(3)]
        us = [dom.field(l, "u")[:, 0].copy() for l in range(3)]
        runs[storage] = dict(hist_ms=ev[0].elapsed_time(ev[1]), solve_ms=solve_ms, us=us, energy=e,
                             total_ms=ev[0].elapsed_time(ev[6]))
        dom.close()
    nv = [d.nvox for d in L]
    pairs = sum(nv) * len(sc["cameras"])
    out = {}
    for storage, r in runs.items():
        upd = sum(n * iters for n in nv)
        out[storage] = {"voxel_updates_per_s": upd / (sum(r["solve_ms"]) / 1e3),
                        "solve_ms_per_level": r["solve_ms"], "histogram_ms": r["hist_ms"],
                        "voxel_map_pairs_per_s": pairs / (r["hist_ms"] / 1e3), "total_ms": r["total_ms"],
                        "gap_level2": r["energy"][2], "certified": bool(r["energy"][3])}
        if storage != "fp32":
            out[storage]["u_err_inf_vs_fp32_per_level"] = [float(np.max(np.abs(a - b))) for a, b in
                                                            zip(r["us"], runs["fp32"]["us"])]
    return {"metric": "multilevel coarse-to-fine: voxel-updates/s (3 levels, 200 iterations each)",
            "value": out["fp32"]["voxel_updates_per_s"], "unit": "voxel-updates/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded terrain + blob scene)",
            "config": {"workload": "sparse-3-level-terrain+blob-256x1024^2-maps-10bins-200it",
                       "active_voxels_per_level": nv, "frozen_bricks_per_level": [d.nfrozen for d in L],
                       "maps": len(sc["cameras"]), "generation_s": t_gen},
            "runs": out,
            "accuracy_note": "16-bit storage error vs the FP32 run at full size; vs the FP64 oracle on the "
                             "scaled-down scene in tests/test_gpu_multilevel.py"}


def _dense_zyx(vals, bricks, n):
    """Per-voxel values (brick order, x fastest in a brick) on an (n, n, n) [z, y, x] grid."""
    li = np.arange(512)
    loc = np.stack([li % 8, (li // 8) % 8, li // 64], axis=1)
    g = (8 * np.asarray(bricks)[:, None, :] + loc[None]).reshape(-1, 3)
    out = np.zeros((n, n, n), dtype=np.float64)
    out[g[:, 2], g[:, 1], g[:, 0]] = np.asarray(vals, np.float64).reshape(-1)
    return out


def _field_diff(U, R, eps=1e-3, votes=None):
    """Differences of field U against the reference R on one grid: max and RMS of |U - R|,
    and on voxel edges whose endpoints have |value| > eps in both fields: the share of
    edges where the sign pattern differs and the displacement of the zero crossing
    (linear interpolation, in voxel edges h) where both cross.  With `votes` (per-voxel
    vote totals on the grid) the crossing displacement is also given over the observed
    edges (both end voxels with >= 2 votes)."""
    d = U - R
    out = {"linf": float(np.abs(d).max()), "rms": float(np.sqrt(np.mean(d * d)))}
    n_edges = n_mismatch = 0
    disp, disp_obs = [], []
    for ax in range(3):
        s0 = [slice(None)] * 3
        s1 = [slice(None)] * 3
        s0[ax] = slice(0, -1)
        s1[ax] = slice(1, None)
        ua, ub, ra, rb = U[tuple(s0)], U[tuple(s1)], R[tuple(s0)], R[tuple(s1)]
        ok = (np.abs(ua) > eps) & (np.abs(ub) > eps) & (np.abs(ra) > eps) & (np.abs(rb) > eps)
        cu = np.sign(ua) != np.sign(ub)
        cr = np.sign(ra) != np.sign(rb)
        n_edges += int(np.count_nonzero(ok & (cu | cr)))
        n_mismatch += int(np.count_nonzero(ok & (cu != cr)))
        both = ok & cu & cr
        tu = ua[both] / (ua[both] - ub[both])
        tr = ra[both] / (ra[both] - rb[both])
        disp.append(np.abs(tu - tr))
        if votes is not None:
            obs = ((votes[tuple(s0)] >= 2) & (votes[tuple(s1)] >= 2))[both]
            disp_obs.append(np.abs(tu - tr)[obs])
    disp = np.concatenate(disp)
    if votes is not None:
        dob = np.concatenate(disp_obs)
        out["observed"] = {"linf": float(np.abs(d[votes >= 2]).max()), "crossing_edges": int(len(dob)),
                           "crossing_disp_max_h": float(dob.max()) if len(dob) else 0.0}
    out.update({"crossing_edges": n_edges, "sign_mismatch_share": n_mismatch / max(n_edges, 1),
                "crossing_disp_max_h": float(disp.max()) if len(disp) else 0.0,
                "crossing_disp_mean_h": float(disp.mean()) if len(disp) else 0.0})
    return out


def run_precision(args):
    """Reduced-precision storage of v, vbar, p, q against FP32 and the FP64 oracle: max and
    RMS difference of u and the displacement of its zero crossings, on the sphere case
    (64^3, 16 maps, 200 iterations; against the oracle) and the terrain case (256^3, 64
    maps, 500 iterations; against the FP32 run)."""
    import torch
    import synth
    import oracle
    from paper_2107_14790_b300 import build, tgv
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    res = {}
    sph = synth.sphere_scene()
    # cpu_baseline leg: the oracle's run of the sphere case, timed; its field is the reference
    t_cpu = time.perf_counter()
    orc = oracle.OracleLevel(sph.domain, 8)
    for c, d in zip(sph.cameras, sph.depths):
        orc.accumulate(c, d, 1)
    orc.iterate(200)
    t_cpu = time.perf_counter() - t_cpu
    n1 = 64
    ref1 = _dense_zyx(orc.u, sph.domain.bricks, n1)
    dep1 = torch.from_numpy(np.stack(sph.depths)).cuda()
    sc = synth.terrain_scene(1002, 256, 64, 512, 10, 500, device="cuda")
    dep2 = torch.from_numpy(np.stack(sc.depths)).cuda()
    ref2 = None
    votes1 = _dense_zyx(orc.hist.sum(1), sph.domain.bricks, n1)
    votes2 = None
    for storage in ("fp32", "fx16", "fp16", "bf16"):
        with tgv.Domain([sph.domain], nbins=8, storage=storage, stream=stream.cuda_stream) as dom:
            dom.accumulate(0, sph.cameras, dep1)
            dom.solve(0, 200)
            u1 = _dense_zyx(dom.field(0, "u")[:, 0], sph.domain.bricks, n1)
        with tgv.Domain([sc.domain], nbins=10, storage=storage, stream=stream.cuda_stream) as dom:
            dom.accumulate(0, sc.cameras, dep2)
            if votes2 is None:
                votes2 = _dense_zyx(dom.histograms(0).sum(1), sc.domain.bricks, 256)
            dom.solve(0, 500)
            u2 = _dense_zyx(dom.field(0, "u")[:, 0], sc.domain.bricks, 256)
        if storage == "fp32":
            ref2 = u2
        res[storage] = {"sphere_64_vs_fp64_oracle": _field_diff(u1, ref1, votes=votes1),
                        "terrain_256_vs_fp32": _field_diff(u2, ref2, votes=votes2) if storage != "fp32" else None}
    return {"metric": "precision of reduced storage: |du| max / RMS and zero-crossing displacement",
            "value": res["fx16"]["terrain_256_vs_fp32"]["linf"], "unit": "max |u_fx16 - u_fp32| (terrain)",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f32-math/fx16,fp16,bf16-storage",
            "data": "synthetic (seeded sphere and terrain scenes)",
            "config": {"workload": "sphere-64^3-200it-vs-oracle+terrain-256^3-500it-vs-fp32"}, "results": res,
            "cpu_baseline": {"value": sph.domain.nvox * 200 / t_cpu, "unit": "voxel-updates/s",
                             "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": "the sphere case whole (16 maps' histograms + 200 iterations)"}}


def run_histforms(args):
    """The two forms of the histogram kernel on the 256^3 terrain's 64 aerial maps 512^2:
    gather (one thread per voxel, every map) and scatter (one thread per pyramid pixel,
    atomic votes).  Same counts bit for bit (checked here on the whole domain); the time
    of one accumulate call of all 64 maps (pyramids included), CUDA events."""
    import torch
    import synth
    from paper_2107_14790_b300 import build, tgv
    build.build()
    torch.cuda.set_device(0)
    sc = synth.terrain_scene(1002, 256, 64, 512, 10, 500, device="cuda")
    photos = torch.from_numpy(np.stack(sc.depths)).cuda()
    stream = torch.cuda.Stream()
    out = {}
    hists = {}
    for form in ("gather", "scatter"):
        dom = tgv.Domain([sc.domain], nbins=10, stream=stream.cuda_stream, hist_form=form)
        nvox = dom.voxels(0)
        for _ in range(max(1, args.warmup)):
            dom.reset(0, clear_hist=True)
            dom.accumulate(0, sc.cameras, photos)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(args.steps):
            dom.reset(0, clear_hist=True)
            e0.record(stream)
            dom.accumulate(0, sc.cameras, photos)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        hists[form] = dom.histograms(0)
        dom.close()
        med = float(np.median(ms))
        out[form] = {"ms": med, "pairs_per_s": nvox * len(sc.cameras) / (med / 1e3)}
    same = bool(np.array_equal(hists["gather"], hists["scatter"]))
    return {"metric": "histograms: (voxel, map) pairs/s (Alg. 1), gather vs scatter form",
            "value": out["scatter"]["pairs_per_s"], "unit": "pairs/s", "n_gpus": 1, "higher_is_better": True,
            "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
            "data": "synthetic (seeded terrain, 64 aerial maps 512^2)",
            "config": {"workload": "dense-256^3-terrain-64x512^2-maps-10bins-histograms", "voxels": nvox,
                       "maps": len(sc.cameras)},
            "gather": out["gather"], "scatter": out["scatter"],
            "scatter_over_gather": out["scatter"]["pairs_per_s"] / out["gather"]["pairs_per_s"],
            "votes_total": int(hists["gather"].sum()), "identical_counts": same}


def run_lidar(args):
    """Ground LIDAR scans (spherical range maps, vote 5) of the 256^3 terrain next to its 64
    aerial photos (pinhole z-depth maps, vote 1): histogram throughput of each map kind, then
    the whole step (both kinds of maps + 500 fused iterations + 20 energy/gap evaluations);
    a sample of bricks checked bit for bit against the oracle."""
    import torch
    import synth
    from paper_2107_14790_b300 import build, tgv
    build.build()
    torch.cuda.set_device(0)
    t_gen = time.perf_counter()
    sc = synth.terrain_scene(1002, 256, 64, 512, 10, 500, device="cuda")
    scans, ranges = synth.terrain_lidar_scans(sc.meta["terrain"], nscans=16, width=2048, height=1024, device="cuda")
    t_gen = time.perf_counter() - t_gen
    photos = torch.from_numpy(np.stack(sc.depths)).cuda()
    lidar = torch.from_numpy(np.stack(ranges)).cuda()
    votes5 = [5] * len(scans)
    stream = torch.cuda.Stream()
    dom = tgv.Domain([sc.domain], nbins=10, stream=stream.cuda_stream)
    nvox = dom.voxels(0)

    def timed(fn, reps):
        for _ in range(max(1, args.warmup)):
            dom.reset(0, clear_hist=True)
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(reps):
            dom.reset(0, clear_hist=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / reps

    ms_lidar = timed(lambda: dom.accumulate(0, scans, lidar, votes5), args.steps)
    ms_photo = timed(lambda: dom.accumulate(0, sc.cameras, photos), args.steps)

    def step():
        dom.accumulate(0, sc.cameras, photos)
        dom.accumulate(0, scans, lidar, votes5)
        for _ in range(20):
            dom.solve(0, 25)
            tgv.tgv_energy(dom.handle, 0)

    ms_step = timed(step, args.steps)
    dom.reset(0, clear_hist=True)
    dom.accumulate(0, sc.cameras, photos)
    dom.accumulate(0, scans, lidar, votes5)
    h_gpu = dom.histograms(0)
    e = dom.energy(0)
    dom.close()
    # CPU baseline: the oracle's Alg. 1 on 48 sampled bricks with all 80 maps (timed),
    # whose counts also serve as a bit-exact check of the same bricks
    import oracle
    rng = np.random.default_rng(7)
    pick = np.sort(rng.choice(sc.domain.nbricks, 48, replace=False))
    sub = synth.DomainDesc(sc.domain.origin, sc.domain.h, sc.domain.bricks[pick])
    orc = oracle.OracleLevel(sub, 10)
    t_cpu = time.perf_counter()
    for c, d in zip(scans, ranges):
        orc.accumulate(c, d, 5)
    t_cpu = time.perf_counter() - t_cpu
    for c, d in zip(sc.cameras, sc.depths):
        orc.accumulate(c, d, 1)
    rows = (pick[:, None] * 512 + np.arange(512)[None, :]).ravel()
    mism = int(np.count_nonzero(h_gpu[rows] != orc.hist))
    lidar_pairs = nvox * len(scans)
    return {"metric": "LIDAR histograms: (voxel, spherical map) pairs/s (Alg. 1, vote 5)",
            "value": lidar_pairs / (ms_lidar / 1e3), "unit": "pairs/s", "n_gpus": 1, "higher_is_better": True,
            "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
            "data": "synthetic (seeded terrain, 16 ground scans 2048x1024 + 64 aerial photos 512^2)",
            "config": {"workload": "dense-256^3-terrain-16-lidar-scans-2048x1024-64-photos-512^2-10bins-500it",
                       "voxels": nvox, "scans": len(scans), "photos": len(sc.cameras), "generation_s": t_gen},
            "lidar_histogram_ms": ms_lidar, "photo_histogram_ms": ms_photo,
            "photo_pairs_per_s": nvox * len(sc.cameras) / (ms_photo / 1e3),
            "votes_total": int(h_gpu.sum()), "step_ms": ms_step,
            "step_voxel_updates_per_s": nvox * 500 / (ms_step / 1e3),
            "energy_gap": {"energy": e[0], "gap": e[2], "certified": bool(e[3])},
            "cpu_baseline": {"value": 48 * 512 * len(scans) / t_cpu, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                             "sample": "48 random bricks x 16 LIDAR scans (its pyramids included)"},
            "parity_sample": {"bricks": int(len(pick)), "maps": len(scans) + len(sc.cameras),
                              "mismatched_counts": mism}}


def run_mesh(args):
    """Marching cubes (Sec. 4.6) of the solved 256^3 terrain field (64 maps, 10 bins, 500
    iterations): cells/s and triangles/s of the extraction (count pass, scans, write pass,
    with the device-to-host copy of the mesh timed separately)."""
    import torch
    import synth
    from paper_2107_14790_b300 import build, tgv
    build.build()
    torch.cuda.set_device(0)
    sc = synth.terrain_scene(1002, 256, 64, 512, 10, 500, device="cuda")
    stream = torch.cuda.Stream()
    dom = tgv.Domain([sc.domain], nbins=10, stream=stream.cuda_stream)
    dom.accumulate(0, sc.cameras, torch.from_numpy(np.stack(sc.depths)).cuda())
    dom.solve(0, 500)
    dom.synchronize()
    import ctypes
    cv, ct = ctypes.c_int64(0), ctypes.c_int64(0)
    for _ in range(max(1, args.warmup)):
        tgv._check(dom.handle, tgv.lib().tgv_extract_mesh(dom.handle, 0, ctypes.byref(cv), ctypes.byref(ct)))
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        tgv._check(dom.handle, tgv.lib().tgv_extract_mesh(dom.handle, 0, ctypes.byref(cv), ctypes.byref(ct)))
        times.append(time.perf_counter() - t0)
    nv, nt = cv.value, ct.value
    verts = np.zeros((nv, 3), np.float32)
    tris = np.zeros((nt, 3), np.int32)
    t0 = time.perf_counter()
    tgv.tgv_copy_mesh(dom.handle, verts, tris)
    t_copy = time.perf_counter() - t0
    ncell = dom.voxels(0)
    dom.close()
    t = float(np.median(times))
    # open surface (it leaves the domain), but every interior edge must have its reverse
    key = lambda a, b: a.astype(np.int64) * (1 << 32) + b
    e = np.concatenate([key(tris[:, 0], tris[:, 1]), key(tris[:, 1], tris[:, 2]), key(tris[:, 2], tris[:, 0])])
    r = np.concatenate([key(tris[:, 1], tris[:, 0]), key(tris[:, 2], tris[:, 1]), key(tris[:, 0], tris[:, 2])])
    dup = len(e) - len(np.unique(e))
    unpaired = int(np.count_nonzero(~np.isin(e, r)))
    return {"metric": "marching cubes: cells/s (zero level set of the solved field, Sec. 4.6)",
            "value": ncell / t, "unit": "cells/s", "n_gpus": 1, "higher_is_better": True, "steps": args.steps,
            "warmup": args.warmup, "dtype": "f32", "data": "synthetic (seeded terrain scene, 64 maps, 500 iterations)",
            "config": {"workload": "dense-256^3-terrain-solved-500it-marching-cubes", "cells": ncell},
            "extract_ms": t * 1e3, "copy_to_host_ms": t_copy * 1e3, "vertices": nv, "triangles": nt,
            "triangles_per_s": nt / t, "repeated_directed_edges": dup, "edges_without_reverse": unpaired,
            "note": "edges without a reverse lie on the domain boundary, where the surface is cut"}


def run_octree(args):
    """Brick domain from the 64 terrain maps (512^2) by Eq. 4 (depths 5..9 of the unit root
    cube, band 1, 2:1 balance, frozen shells): samples/s of the whole build, timed as the
    library call (it synchronises); the oracle's build of the same maps as CPU baseline and
    as a bit-exact check of every level; then the same build from 16 ground LIDAR scans."""
    import torch
    import synth
    from paper_2107_14790_b300 import build, tgv
    build.build()
    torch.cuda.set_device(0)
    sc = synth.terrain_scene(1002, 256, 64, 512, 10, 500, device="cuda")
    depth = torch.from_numpy(np.stack(sc.depths)).cuda()
    stream = torch.cuda.Stream()
    cfgs = (np.zeros(3), 1.0, 5, 9, 1)
    for _ in range(max(1, args.warmup)):
        tgv.tgv_octree_build(sc.cameras, depth, *cfgs, stream=stream.cuda_stream)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        levels, ns = tgv.tgv_octree_build(sc.cameras, depth, *cfgs, stream=stream.cuda_stream)
        times.append(time.perf_counter() - t0)
    t = float(np.median(times))
    import oracle
    t_cpu = time.perf_counter()
    ref, ns_ref = oracle.octree_build(sc.cameras, sc.depths, *cfgs)
    t_cpu = time.perf_counter() - t_cpu
    same = ns == ns_ref and all(np.array_equal(L.bricks, a) and np.array_equal(L.frozen, f)
                                for L, (a, f) in zip(levels, ref))
    # the same build from 16 ground LIDAR scans (spherical range maps 2048 x 1024)
    scans, ranges = synth.terrain_lidar_scans(sc.meta["terrain"], nscans=16, width=2048, height=1024, device="cuda")
    rdev = torch.from_numpy(np.stack(ranges)).cuda()
    tl = []
    for k in range(max(1, args.warmup) + args.steps):
        t0 = time.perf_counter()
        lv_l, ns_l = tgv.tgv_octree_build(scans, rdev, *cfgs, stream=stream.cuda_stream)
        if k >= max(1, args.warmup):
            tl.append(time.perf_counter() - t0)
    ref_l, ns_l_ref = oracle.octree_build(scans, ranges, *cfgs)
    same_l = ns_l == ns_l_ref and all(np.array_equal(L.bricks, a) and np.array_equal(L.frozen, f)
                                      for L, (a, f) in zip(lv_l, ref_l))
    lidar = {"scans": len(scans), "size": "2048x1024", "samples": ns_l, "build_ms": 1e3 * float(np.median(tl)),
             "samples_per_s": ns_l / float(np.median(tl)), "identical_to_oracle": bool(same_l),
             "levels": [{"depth": 5 + l, "active": L.nbricks, "frozen": L.nfrozen} for l, L in enumerate(lv_l)]}
    return {"metric": "octree domain build: depth samples/s (Eq. 4, Sec. 4.1-4.2)", "value": ns / t,
            "unit": "samples/s", "n_gpus": 1, "higher_is_better": True, "steps": args.steps, "warmup": args.warmup,
            "dtype": "f32", "data": "synthetic (seeded terrain scene, 64 maps 512^2)",
            "config": {"workload": "terrain-64x512^2-maps-octree-depths-5..9-band1", "samples": ns},
            "build_ms": t * 1e3,
            "levels": [{"depth": 5 + l, "active": L.nbricks, "frozen": L.nfrozen} for l, L in enumerate(levels)],
            "cpu_baseline": {"value": ns_ref / t_cpu, "unit": "samples/s", "cores": 1, "kind": "oracle",
                             "sample": "the whole build of the same maps"},
            "identical_to_oracle": bool(same), "lidar": lidar}


def run_composite(args):
    """Joint solve across levels on the composite grid (2:1 faces): the 5 octree levels built
    from the 64 terrain maps (depths 5..9, band 1), Alg. 1 histograms on every level, then
    joint iterations (dual kernel + primal kernel per iteration over every leaf); the treetop
    of the leaves (wall time of the library call)."""
    import torch
    import synth
    from paper_2107_14790_b300 import build, tgv
    build.build()
    torch.cuda.set_device(0)
    sc = synth.terrain_scene(1002, 256, 64, 512, 10, 500, device="cuda")
    depth = torch.from_numpy(np.stack(sc.depths)).cuda()
    stream = torch.cuda.Stream()
    lv, _ = tgv.tgv_octree_build(sc.cameras, depth, np.zeros(3), 1.0, 5, 9, 1, stream=stream.cuda_stream)
    levels = [synth.DomainDesc(L.origin, L.h, L.bricks) for L in lv]
    iters = 100
    dom = tgv.Domain(levels, nbins=10, stream=stream.cuda_stream)
    for l in range(len(levels)):
        dom.accumulate(l, sc.cameras, depth)
    t0 = time.perf_counter()
    comp = tgv.Composite(dom)
    t_build = time.perf_counter() - t0
    comp.solve(5)
    dom.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(args.steps):
        e0.record(stream)
        comp.solve(iters)
        e1.record(stream)
        dom.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    n = comp.leaves
    per_level = [comp.level_leaves(l) for l in range(len(levels))]
    # treetop (Sec. 4.3) of the leaf cubes: root = the octree root, voxel depth 9 + 3
    # (wall time of tgv_composite_treetop, which synchronises; the parts copied afterwards)
    import ctypes
    treetop = {}
    for N in (1 << 24, 1 << 20):
        tt, nparts = [], ctypes.c_int64(0)
        for _ in range(4):
            t0 = time.perf_counter()
            tgv._check(dom.handle, tgv.lib().tgv_composite_treetop(comp.handle, 12, N, ctypes.byref(nparts)))
            tt.append(time.perf_counter() - t0)
        dpt, _, first, last, _ = tgv.tgv_composite_treetop_parts(comp.handle, dom.handle, nparts.value)
        treetop[f"N=2^{N.bit_length() - 1}"] = {"parts": int(len(dpt)), "ms": 1e3 * float(np.median(tt[1:])),
                                                 "largest_part": int(np.max(last - first + 1)),
                                                 "depths": sorted(set(int(x) for x in dpt))}
    comp.close()
    dom.close()
    bpl = 192  # state bytes per leaf-update (dual: read 13, write 9 floats; primal: read 13 + hist, write 8)
    peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6400.0
    achieved = n * bpl / (ms / 1e3 / iters) / 1e9
    # CPU baseline: the oracle's composite iteration on the two coarsest levels (timed)
    import oracle
    from oracle.composite import Composite as OC
    small = OC([L.bricks for L in levels[:2]], 10)
    t_cpu = time.perf_counter()
    small.iterate(5)
    t_cpu = time.perf_counter() - t_cpu
    return {"metric": "joint multilevel solve: leaf-updates/s (composite grid over 2:1 faces)",
            "value": n * iters / (ms / 1e3), "unit": "leaf-updates/s", "n_gpus": 1, "higher_is_better": True,
            "steps": args.steps, "dtype": "f32", "data": "synthetic (seeded terrain scene, 64 maps 512^2)",
            "config": {"workload": "terrain-octree-depths-5..9-composite-100it", "leaves": n,
                       "leaves_per_level": per_level},
            "ms_per_100_iterations": ms, "build_s": t_build,
            "treetop": treetop,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "algorithmic_bytes_per_leaf": bpl,
                         "note": "state bytes only; regular leaves add 24 B of neighbour ids, leaves at 2:1 faces 192 B of lists"},
            "cpu_baseline": {"value": small.n * 5 / t_cpu, "unit": "leaf-updates/s", "cores": 1, "kind": "oracle",
                             "sample": f"composite of the two coarsest levels ({small.n} leaves), 5 iterations"}}


def run_serving(args):
    """Poisson stream of chunk-solve requests (16k..8M voxels, 8..12 bins, 200..600 iterations)
    through one server per bin count, arenas sized from the HBM budget; plus an overload run."""
    import torch
    from paper_2107_14790_b300 import build
    build.build()
    torch.cuda.set_device(0)
    r = serving_block(args.storage, args.requests, args.budget_gb, overload=min(args.requests, 400))
    r.pop("latencies")
    return {"metric": "chunk-solve serving: p50/p99 latency and voxel-updates/s (Poisson arrivals, 0.8x saturated rate)",
            "value": r["voxel_updates_per_s"], "unit": "voxel-updates/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32" if args.storage == "fp32" else f"f32-math/{args.storage}-storage",
            "data": "synthetic (seeded chunk requests)",
            "config": {"workload": "serving-%d-requests-16k..8M-voxels-8..12bins-200..600it" % args.requests,
                       "requests": args.requests, "budget_gb": args.budget_gb, "servers": r["servers"],
                       "round_iterations": 10},
            "serving": r}


def main():
    args = parse()
    from paper_2107_14790_b300.multigpu import launched_as_rank, relaunch
    if args.gpus > 1 and not launched_as_rank():
        # one process per GPU: start `--gpus` ranks of this same command under torch.distributed.run
        sys.exit(relaunch(args.gpus, os.path.abspath(__file__), sys.argv[1:]))
    if args.profile:
        run_profile_case(args)
        return
    if args.workload == "batched":
        res = run_batched(args)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if args.workload == "serving":
        print(json.dumps(run_serving(args)), flush=True)
        return
    if args.workload == "multilevel":
        print(json.dumps(run_multilevel(args)), flush=True)
        return
    if args.workload == "composite":
        print(json.dumps(run_composite(args)), flush=True)
        return
    if args.workload == "octree":
        print(json.dumps(run_octree(args)), flush=True)
        return
    if args.workload == "mesh":
        print(json.dumps(run_mesh(args)), flush=True)
        return
    if args.workload == "lidar":
        print(json.dumps(run_lidar(args)), flush=True)
        return
    if args.workload == "histforms":
        print(json.dumps(run_histforms(args)), flush=True)
        return
    if args.workload == "precision":
        print(json.dumps(run_precision(args)), flush=True)
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
