#!/usr/bin/env python3
"""Benchmark of whole multi-scale registrations (Algorithm 1) on the
brain-MRI-shaped synthetic pair: 160x192x224 Voronoi volumes, scales
{4, 2, 1} x iterations {200, 100, 50}, LNCC window 5, lr 0.5,
sigma_grad 1, sigma_warp 0.5.  One step = one whole registration of one pair
(pyramid, all levels, final loss) with the inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode fused|plain]
    python bench.py --impl reference     # the FP64 oracle on the host cores

Prints one JSON line (rank 0).  Under torchrun each rank registers its own
pair (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(name="voronoi_brain_160x192x224", shape=(160, 192, 224), scales=(4, 2, 1),
                iters=(200, 100, 50), window=5, lr=0.5, sigma_grad=1.0, sigma_warp=0.5,
                cc_eps=1e-5)
METRIC = "voxel-iters/s"
L2_BYTES = 129 * 1024 * 1024
HBM_FALLBACK_GBS = 6800.0
# algorithmic bytes per voxel of one launch of each timed kernel: every input
# field read once, every output field written once (fp32 storage, S_I int64)
ALGO_BYTES = {
    "fused_warp_lncc": 4 + 4 + 8 + 4 + 16,      # I_f, J, S_I, var_I read; A, B, C hi/lo written
    "fused_lncc_grad": 16 + 12 + 4 + 4 + 12,    # A, B, C hi/lo, grad I_m(phi), I_f, J read; g written
    "fused_smooth_adam": 12 * 3 + 12 * 3,       # g, m, v read; m, v, d written
    "fused_compose": 12 + 12 + 4 + 12 + 4 + 12,  # d, u, I_m read; u', J, grad I_m(phi') written
    "plain_iteration": 80,                      # whole iteration: I_f, I_m, u, m, v once
}
# the whole path per voxel-iteration: read I_f, I_m, u, m, v, write u, m, v
PATH_BYTES = 80
KERNEL_IDS = {"fused_warp_lncc": 0, "fused_lncc_grad": 1, "fused_smooth_adam": 2,
              "fused_compose": 3, "plain_iteration": 4}
FUSED_KERNELS = ("fused_warp_lncc", "fused_lncc_grad", "fused_smooth_adam", "fused_compose")
TIMED_ITERS = 10  # finest-level iterations whose kernels are timed per step


def level_size(n, s):
    return max(1, n // s)


def voxel_iters(shape, scales, iters):
    tot = 0
    for s, t in zip(scales, iters):
        n = 1
        for a in shape:
            n *= level_size(a, s)
        tot += n * t
    return tot


def rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus = (bus_id or "").lower()
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 9]
        rows = [[c.strip() for c in r] for r in rows]
        if not rows:
            return None
        buses = {r[1].lower() for r in rows}
        if len(buses) > 1 and self.bus:
            rows = [r for r in rows if r[1].lower().endswith(self.bus[-12:])] or rows
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# --------------------------------------------------------------- oracle leg
def oracle_sample(f, m, iters: int):
    """Times the FP64 oracle on `iters` finest-level iterations of the pair
    (plus its final-loss evaluation); returns (seconds, voxel-iterations, threads)."""
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.register(f, m, [1], [iters], lr=WORKLOAD["lr"], sigma_grad=WORKLOAD["sigma_grad"],
                    sigma_warp=WORKLOAD["sigma_warp"], window=WORKLOAD["window"],
                    cc_eps=WORKLOAD["cc_eps"])
    dt = time.perf_counter() - t0
    return dt, iters * int(np.prod(f.shape)), int(os.environ["OMP_NUM_THREADS"])


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return 0
    from paper_2404_01249_gb300 import synth
    f, m, _ = synth.voronoi_pair(shape=WORKLOAD["shape"], seed=1000)
    for _ in range(args.warmup):
        oracle_sample(f, m, 1)
    times, units = [], 0
    for _ in range(args.steps):
        dt, vi, threads = oracle_sample(f, m, 1)
        times.append(dt)
        units += vi
    total = sum(times)
    val = units / total
    sample = ("1 finest-level iteration (scale 1, 160x192x224) of the pair plus the oracle's "
              "final-loss evaluation per step")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": METRIC, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, world),
            "cpu_baseline": {"value": val, "unit": METRIC, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict(args, world):
    return {"workload": WORKLOAD["name"], "shape": list(WORKLOAD["shape"]),
            "scales": list(WORKLOAD["scales"]), "iters": list(WORKLOAD["iters"]),
            "window": WORKLOAD["window"], "lr": WORKLOAD["lr"],
            "sigma_grad": WORKLOAD["sigma_grad"], "sigma_warp": WORKLOAD["sigma_warp"],
            "loss": "lncc", "mode": args.mode, "u_storage": args.field,
            "pairs_per_rank": 1, "world_size": world,
            "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}"}


def profile_entry(kernel: str):
    """The committed ncu figures of a fused kernel, if they were taken on the
    current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d[kernel]
        h = hashlib.sha256()
        for name in e["sources"]:  # the kernel's code and the helpers it inlines
            h.update(open(os.path.join(ROOT, "paper_2404_01249_gb300", "csrc", name), "rb").read())
        if h.hexdigest()[:16] != e["sources_sha"]:
            return None
        return e
    except Exception:
        return None


def traffic_from_profile(kernel: str, n_voxels: int):
    """DRAM bytes per launch from the committed ncu summary (None if stale)."""
    e = profile_entry(kernel)
    return None if e is None else float(e["dram_bytes_per_voxel"]) * n_voxels


# instruction issue: 4 schedulers per SM, each issuing one warp instruction
# per clock, on every SM
SMS = 152
ISSUE_PER_SM_CLOCK = 4


def issue_roofline(kernels: dict, n_voxels: int, sm_mhz):
    """Issued warp instructions per second of each fused kernel (the committed
    ncu count per voxel x voxels / the live average launch time) against the
    GPU's issue rate at the SM clock sampled during the run."""
    mhz = sm_mhz if sm_mhz else 2070.0
    peak = SMS * ISSUE_PER_SM_CLOCK * mhz * 1e6
    out = {}
    for kn, k in kernels.items():
        e = profile_entry(kn)
        if e is None or "warp_inst_per_voxel" not in e:
            continue
        rate = float(e["warp_inst_per_voxel"]) * n_voxels / (k["avg_launch_ms"] / 1e3)
        out[kn] = {"warp_inst_per_voxel": float(e["warp_inst_per_voxel"]),
                   "achieved": rate, "frac": round(rate / peak, 4)}
    return {"unit": "warp instructions/s", "peak": peak, "sm_mhz": mhz,
            "peak_from": f"{SMS} SMs x {ISSUE_PER_SM_CLOCK} warp instructions per clock",
            "kernels": out}


def whole_job_rate(local_ms: float, units_per_rank: float, world: int, device) -> tuple:
    """The job's time is the slowest rank's (max over ranks of the local
    time); its rate is the units all ranks processed over that time.
    Returns (max_ms, rate)."""
    ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms / 1e3)


# --------------------------------------------------------------- GPU leg
def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2404_01249_gb300 import build, fa, synth

    rank, world, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    fa.load()
    shape = WORKLOAD["shape"]
    f, m, _ = synth.voronoi_pair(shape=shape, seed=1000 + rank)
    params = fa.RegParams(scales=WORKLOAD["scales"], iters=WORKLOAD["iters"],
                          window=WORKLOAD["window"], lr=WORKLOAD["lr"],
                          sigma_grad=WORKLOAD["sigma_grad"], sigma_warp=WORKLOAD["sigma_warp"],
                          cc_eps=WORKLOAD["cc_eps"], mode=args.mode, field=args.field)
    fixed = torch.from_numpy(f).to(dev)
    moving = torch.from_numpy(m).to(dev)
    ws = fa.workspace(fa.fa_register_workspace_size(shape, params), dev)
    u = torch.empty((3,) + shape, device=dev)
    loss = torch.empty((), device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # tile choices of the fused kernels for this workload (outside any timing)
    tuned = []
    if args.mode == "fused" and not args.no_autotune:
        tuned = fa.fa_autotune(shape, params, ws=ws)

    # kernel timers on the finest level, inside the recorded graph: fused mode
    # times all four fused kernels (launch order K1 K2 K3 K4 per iteration),
    # plain mode the whole plain iteration.  Two timers alternate between
    # steps so that one step's events are read before they are recorded again.
    fin = len(WORKLOAD["scales"]) - 1
    if args.mode == "plain":
        knames, kid = ["plain_iteration"], fa.FA_K_PLAIN_ANY
    else:
        knames, kid = list(FUSED_KERNELS), fa.FA_K_FUSED_ALL
    # the first TIMED_ITERS finest-level iterations (event records between
    # launches interrupt programmatic dependent launch, so not all of them)
    cap = min(WORKLOAD["iters"][fin], TIMED_ITERS) * len(knames)
    timers = []
    for _ in range(2):
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(cap)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(cap)]
        timers.append((fa.make_timer(kid, fin, ev0, ev1), ev0, ev1))
    ktimes = {k: [] for k in knames}

    def harvest(j):
        tm, ev0, ev1 = timers[j]
        for i in range(tm.count):
            ktimes[knames[i % len(knames)]].append(ev0[i].elapsed_time(ev1[i]))

    # warm-up (records the graphs of both timers when W >= 2)
    for w in range(args.warmup):
        fa.fa_register(fixed, moving, params, ws=ws, sync=False, u_out=u, loss_out=loss,
                       timer=timers[w % 2][0])
    torch.cuda.synchronize()
    step0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    step1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    bus = None
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id  # type: ignore[attr-defined]
    except Exception:
        pass
    clocks = ClockSampler(str(bus) if bus is not None else None)

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = fa.fa_launch_count()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        step0[k].record(stream)
        fa.fa_register(fixed, moving, params, ws=ws, sync=False, u_out=u, loss_out=loss,
                       timer=timers[k % 2][0])
        step1[k].record(stream)
        if k >= 1:  # step k is queued: read step k-1's kernel events
            step1[k - 1].synchronize()
            harvest((k - 1) % 2)
    torch.cuda.synchronize()
    harvest((args.steps - 1) % 2)
    wall = time.perf_counter() - t0
    launches = fa.fa_launch_count() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    fa.fa_ws_status(ws)
    step_ms = [a.elapsed_time(b) for a, b in zip(step0, step1)]
    vi = voxel_iters(shape, WORKLOAD["scales"], WORKLOAD["iters"])
    total_ms, value = whole_job_rate(sum(step_ms), vi * args.steps, world, dev)

    # Roofline of the finest-level iteration: the whole path's algorithmic
    # bytes (read I_f, I_m, u, m, nu and write u, m, nu once: 80 B per voxel)
    # over the summed average launch times of the iteration's kernels, timed
    # with CUDA events inside the recorded graph.  Each kernel's own
    # input+output bytes (its intermediates included) give kernel_io_frac.
    n_fine = int(np.prod([level_size(a, WORKLOAD["scales"][fin]) for a in shape]))
    peak, peak_kind = measured_peak()
    kernels = {}
    for kn, kt in ktimes.items():
        if not kt:
            continue
        avg_ms = float(np.mean(kt))
        algo = ALGO_BYTES[kn] * n_fine
        achieved = algo / (avg_ms / 1e3) / 1e9
        kernels[kn] = {"avg_launch_ms": avg_ms, "launches_timed": len(kt), "io_bytes": algo,
                       "achieved": achieved, "frac": achieved / peak,
                       "traffic": traffic_from_profile(kn, n_fine)}
    iter_ms = float(sum(k["avg_launch_ms"] for k in kernels.values()))
    iter_algo = PATH_BYTES * n_fine
    iter_achieved = iter_algo / (iter_ms / 1e3) / 1e9
    traffics = [k["traffic"] for k in kernels.values()]
    iter_traffic = None if any(t is None for t in traffics) else float(sum(traffics))
    dom = max(kernels, key=lambda k: kernels[k]["avg_launch_ms"])
    roofline = {"bound": "hbm", "kernel": "finest_level_iteration",
                "kernels": list(kernels), "achieved": iter_achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": iter_achieved / peak,
                "traffic": iter_traffic, "algo_bytes": iter_algo,
                "algo_bytes_per_voxel_iter": PATH_BYTES, "voxels": n_fine,
                "iteration_ms": iter_ms,
                "traffic_ratio": (None if iter_traffic is None else iter_traffic / iter_algo),
                "dominant_kernel": {"name": dom,
                                    "avg_launch_ms": kernels[dom]["avg_launch_ms"],
                                    "launches_timed": kernels[dom]["launches_timed"]},
                "kernel_io_frac": {k: {"avg_launch_ms": round(v["avg_launch_ms"], 4),
                                       "io_bytes_per_voxel": ALGO_BYTES[k],
                                       "frac": round(v["frac"], 4)}
                                   for k, v in kernels.items()},
                "path": {"bytes_per_voxel_iter": PATH_BYTES,
                         "achieved": PATH_BYTES * vi * args.steps / (total_ms / 1e3) / 1e9,
                         "frac": PATH_BYTES * vi * args.steps / (total_ms / 1e3) / 1e9 / peak}}

    # end to end: host buffers in, displacement and loss out
    fh = torch.from_numpy(f).pin_memory()
    mh = torch.from_numpy(m).pin_memory()
    uh = torch.empty((3,) + shape, dtype=torch.float32).pin_memory()
    lh = torch.empty((), dtype=torch.float32).pin_memory()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    fd = torch.empty_like(fixed)
    md = torch.empty_like(moving)
    fd.copy_(fh)
    md.copy_(mh)
    fa.fa_register(fd, md, params, ws=ws, sync=False, u_out=u, loss_out=loss)  # records its graph
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0.record(stream)
    for _ in range(args.steps):
        fd.copy_(fh, non_blocking=True)
        md.copy_(mh, non_blocking=True)
        fa.fa_register(fd, md, params, ws=ws, sync=False, u_out=u, loss_out=loss)
        uh.copy_(u, non_blocking=True)
        lh.copy_(loss, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    _, e2e_rate = whole_job_rate(e0.elapsed_time(e1), vi * args.steps, world, dev)
    e2e = {"value": e2e_rate, "unit": METRIC,
           "h2d_bytes_per_step": 2 * f.nbytes, "d2h_bytes_per_step": uh.numel() * 4 + 4,
           "final_lncc": -float(lh)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "s_per_pair": total_ms / args.steps / 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(config_dict(args, world),
                               tiles=("autotuned" if tuned else "default"),
                               tile_choices=tuned),
                "wall_s": wall, "roofline": roofline,
                "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
                "final_lncc": -float(loss)}
        if args.mode == "fused":
            roofline["issue"] = issue_roofline(kernels, n_fine, (clk or {}).get("sm_mhz"))
        if world == 1 and not args.no_cpu_baseline:
            dt, units, threads = oracle_sample(f, m, args.cpu_iters)
            line["cpu_baseline"] = {
                "value": units / dt, "unit": METRIC, "cores": threads, "kind": "oracle",
                "sample": f"{args.cpu_iters} finest-level iteration(s) (scale 1, 160x192x224) "
                          "of the same pair plus the oracle's final-loss evaluation"}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------- batched throughput
def _voronoi_pair_job(shape, seed):
    from paper_2404_01249_gb300 import synth
    return synth.voronoi_pair(shape=shape, seed=seed)


def run_batched(args):
    """Throughput of many independent registrations: `--batched P` pairs of
    uneven brain-like grids (each axis uniform in [96,192] x [112,224] x
    [96,192]) x 9 parameter sets (lr {0.25, 0.5, 1} x sigma_grad {0.5, 1, 2}),
    scales {4,2,1} x iterations {200,100,50}.  A step is the whole batch.
    `--schedule` picks the timed form: lockstep (every iteration one launch
    per fused kernel over all jobs of a wave, fa_register_batched_lockstep),
    streams (fused registrations on `--concurrency` forked streams,
    fa_register_batched) or plain (the per-op schedule on forked streams).
    The other two forms are timed once each on the same batch for
    comparison, with the mean |final loss difference| against the timed form."""
    import torch
    from paper_2404_01249_gb300 import build, fa, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    fa.load()
    shapes = synth.uneven_shapes(n=args.batched, seed=3000)
    # the host-side generator takes seconds per pair: a spawn pool (no CUDA
    # state is inherited) draws the pairs in parallel, same seeds as one by one
    import multiprocessing as mp
    workers = max(1, min(len(shapes), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        pairs = pool.starmap(_voronoi_pair_job, [(sh, 1000 + i) for i, sh in enumerate(shapes)])
    img_dtype = torch.bfloat16 if args.storage == "bf16" else torch.float32
    fixed = [torch.from_numpy(p[0]).to(dev).to(img_dtype) for p in pairs]
    moving = [torch.from_numpy(p[1]).to(dev).to(img_dtype) for p in pairs]

    def cfgs(mode):
        # an FP16 u is a fused-schedule option: the per-op form keeps u in FP32
        field = args.field if mode == "fused" else "f32"
        return [fa.RegParams(scales=WORKLOAD["scales"], iters=WORKLOAD["iters"], lr=lr,
                             sigma_grad=sg, sigma_warp=WORKLOAD["sigma_warp"],
                             window=WORKLOAD["window"], mode=mode, state=args.storage,
                             field=field)
                for lr in (0.25, 0.5, 1.0) for sg in (0.5, 1.0, 2.0)]

    n_cfg = len(cfgs("fused"))
    vi = sum(voxel_iters(sh, WORKLOAD["scales"], WORKLOAD["iters"]) for sh in shapes) * n_cfg
    n_jobs = len(shapes) * n_cfg
    waves = -(-n_jobs // 64)
    wave = -(-n_jobs // waves)  # balanced waves of at most 64 jobs
    forms = {
        "lockstep": lambda: fa.fa_register_batched_lockstep(fixed, moving, cfgs("fused"),
                                                            jobs_per_wave=wave, sync=False),
        "streams": lambda: fa.fa_register_batched(fixed, moving, cfgs("fused"),
                                                  concurrency=args.concurrency, sync=False),
        "plain": lambda: fa.fa_register_batched(fixed, moving, cfgs("plain"),
                                                concurrency=args.concurrency, sync=False),
    }
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(form, steps):
        e0.record(stream)
        out = None
        for _ in range(steps):
            out = forms[form]()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, out

    for _ in range(args.warmup):
        forms[args.schedule]()
    torch.cuda.synchronize()
    n0 = fa.fa_launch_count()
    clocks = ClockSampler(None)
    clocks.start()
    ms, out = timed(args.schedule, args.steps)
    clk = clocks.stop()
    launches = (fa.fa_launch_count() - n0) // max(args.steps, 1)
    loss = torch.stack([r["loss"] for r in out]).cpu().numpy()
    others = {}
    for form in forms:
        if form == args.schedule or args.no_compare:
            continue
        forms[form]()  # warm (records its graphs)
        torch.cuda.synchronize()
        ms_o, out_o = timed(form, 1)
        lo = torch.stack([r["loss"] for r in out_o]).cpu().numpy()
        others[form] = {"ms_per_step": ms_o, "speedup_of_timed_form": ms_o / ms,
                        "mean_abs_final_loss_diff": float(np.abs(lo - loss).mean()),
                        "max_abs_final_loss_diff": float(np.abs(lo - loss).max())}
    line = {"metric": METRIC, "value": vi / (ms / 1e3), "unit": METRIC, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"uneven_brain_batch_{len(shapes)}x{n_cfg}",
                       "schedule": args.schedule, "jobs_per_wave": wave,
                       "storage": (("bf16 images and Adam moments, " if args.storage == "bf16"
                                    else "fp32 images and Adam moments, ")
                                   + ("fp16 displacement (fp32 in the plain form), "
                                      if args.field == "f16" else "fp32 displacement, ")
                                   + "fp32 arithmetic"),
                       "concurrency": args.concurrency,
                       "shapes": [list(x) for x in shapes], "scales": list(WORKLOAD["scales"]),
                       "iters": list(WORKLOAD["iters"]), "lr": [0.25, 0.5, 1.0],
                       "sigma_grad": [0.5, 1.0, 2.0],
                       "l2": "inputs of the batch exceed L2"},
            "registrations_per_s": n_jobs / (ms / 1e3), "s_per_pair": ms / 1e3 / n_jobs,
            "gpu_launches": int(launches), "other_schedules": others, "clocks": clk}
    if not args.no_cpu_baseline:
        dt, units, threads = oracle_sample(pairs[0][0], pairs[0][1], 1)
        line["cpu_baseline"] = {
            "value": units / dt, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": "1 finest-level iteration of the batch's first pair "
                      f"({'x'.join(map(str, shapes[0]))}) plus the oracle's final-loss "
                      "evaluation, scaled to voxel-iters/s (the whole batch would take "
                      f"about {vi / (units / dt) / 3600:.1f} h on these cores)"}
    print(json.dumps(line))
    return 0


# ------------------------------------------------- the other paper workloads
# Whole-path algorithmic bytes per voxel-iteration of each variant: the state
# every iteration must read and write once (FP32), as PATH_BYTES for the main
# path.
VARIANT_BYTES = {
    "symmetric": 8 + 2 * 72,  # I_f, I_m; u, m, nu of both maps read and written
    "inverse": 12 + 72,       # u read; w, m, nu read and written
    "svf": PATH_BYTES,        # I_f, I_m; v, m, nu
    "mi": PATH_BYTES,
    "use_jac": PATH_BYTES,
    "affine": 8,              # I_f, I_m (12 parameters)
    "rigid": 8,
    # 16-bit storage: I_f, I_m, m, nu in BF16 and u in FP16
    "microscopy": 2 + 2 + 6 + 6 + 6 + 6 + 6 + 6,
}
# the expansion-microscopy-shaped pair: 512 x 512 in-plane, 256 planes
MICROSCOPY = dict(shape=(256, 512, 512), scales=(8, 4, 2, 1), iters=(200, 200, 100, 50),
                  window=7)
INVERSE_SCHEDULE = dict(scales=(4, 2, 1), iters=(100, 50, 25))
SYM_INVERSE_SCHEDULE = dict(scales=(2, 1), iters=(50, 25))
SVF_STEPS = 7


def run_variant(args):
    """One of the paper's other workloads on the brain-shaped pair: symmetric
    registration (with its post-hoc inverse), the post-hoc inverse of the
    pair's generating displacement, the SVF (exp) variant, the MI loss, the
    use_jac direction, and the affine and rigid stages; or the
    expansion-microscopy-shaped pair at 256 x 512 x 512 (window 7, scales
    {8,4,2,1} x iterations {200,200,100,50}, BF16 images and moments).  A step is one whole
    call; the same timing rules as the main path (L2 flushed before every
    step, CUDA events, clocks sampled); the oracle is timed on one
    finest-level iteration of the same workload."""
    import torch
    from paper_2404_01249_gb300 import build, fa, synth
    rank, world, local = rank_env()
    if world > 1:
        raise SystemExit("--workload runs on one GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    fa.load()
    w = args.workload
    base = dict(scales=WORKLOAD["scales"], iters=WORKLOAD["iters"], window=WORKLOAD["window"],
                lr=WORKLOAD["lr"], sigma_grad=WORKLOAD["sigma_grad"],
                sigma_warp=WORKLOAD["sigma_warp"], cc_eps=WORKLOAD["cc_eps"])
    if w == "microscopy":
        shape = MICROSCOPY["shape"]
        f, m, psi = synth.microscopy_pair(shape=shape, seed=1000)
        fixed = torch.from_numpy(f).to(dev).bfloat16()
        moving = torch.from_numpy(m).to(dev).bfloat16()
        base.update(scales=MICROSCOPY["scales"], iters=MICROSCOPY["iters"],
                    window=MICROSCOPY["window"])
        cfg = {"workload": "microscopy_cells_256x512x512", "shape": list(shape)}
        vi = voxel_iters(shape, MICROSCOPY["scales"], MICROSCOPY["iters"])
    else:
        shape = WORKLOAD["shape"]
        f, m, psi = synth.voronoi_pair(shape=shape, seed=1000)
        fixed, moving = torch.from_numpy(f).to(dev), torch.from_numpy(m).to(dev)
        cfg = {"workload": f"{w}_voronoi_brain_160x192x224", "shape": list(shape)}
        vi = voxel_iters(shape, WORKLOAD["scales"], WORKLOAD["iters"])
    if w == "symmetric":
        P, Pi = fa.RegParams(**base), fa.RegParams(**SYM_INVERSE_SCHEDULE)
        call = lambda: fa.fa_register_symmetric(fixed, moving, P, Pi, sync=False)["loss"]  # noqa
        cfg.update(base, inverse=SYM_INVERSE_SCHEDULE, loss="lncc")
    elif w == "inverse":
        u = torch.from_numpy(np.ascontiguousarray(psi, dtype=np.float32)).to(dev)
        sched = (INVERSE_SCHEDULE if args.scales is None and args.iters is None else
                 dict(scales=WORKLOAD["scales"], iters=WORKLOAD["iters"]))
        P = fa.RegParams(**sched)
        call = lambda: fa.fa_inverse(u, P, sync=False)["energy"]  # noqa
        vi = voxel_iters(shape, sched["scales"], sched["iters"])
        cfg.update(sched, field="the pair's generating displacement exp(v)")
    elif w == "svf":
        P = fa.RegParams(**base)
        call = lambda: fa.fa_register_svf(fixed, moving, P, steps=SVF_STEPS, sync=False)["loss"]  # noqa
        cfg.update(base, squarings=SVF_STEPS, loss="lncc")
    elif w == "microscopy":
        import ctypes
        P = fa.RegParams(**base, state="bf16", field="f16")
        pc = P.to_c()
        pc.storage = fa.FA_BF16
        ws = fa.workspace(fa.load().fa_register_workspace_size(*shape, ctypes.byref(pc)), dev)
        if not args.no_autotune:
            fa.fa_autotune(shape, P, ws=ws)
        s_last = MICROSCOPY["scales"][-1]
        uo = torch.empty((3,) + tuple(fa.level_size(a, s_last) for a in shape), device=dev)
        lo = torch.empty((), device=dev)
        call = lambda: fa.fa_register(fixed, moving, P, ws=ws, sync=False, u_out=uo, loss_out=lo)["loss"]  # noqa
        cfg.update(base, storage="bf16 images and Adam moments, fp16 displacement, fp32 arithmetic",
                   mode="fused", cells=int(round(1e-3 * np.prod(shape))))
    elif w in ("mi", "use_jac"):
        P = fa.RegParams(**base, loss="mi" if w == "mi" else "lncc", use_jac=(w == "use_jac"))
        ws = fa.workspace(fa.fa_register_workspace_size(shape, P), dev)
        if not args.no_autotune:
            fa.fa_autotune(shape, P, ws=ws)
        uo = torch.empty((3,) + shape, device=dev)
        lo = torch.empty((), device=dev)
        call = lambda: fa.fa_register(fixed, moving, P, ws=ws, sync=False, u_out=uo, loss_out=lo)["loss"]  # noqa
        cfg.update(base, loss=P.loss, use_jac=P.use_jac, mi_bins=P.mi_bins, mode="fused")
    else:  # affine, rigid
        lin = dict(scales=WORKLOAD["scales"], iters=WORKLOAD["iters"], lr=3e-3,
                   window=WORKLOAD["window"], cc_eps=WORKLOAD["cc_eps"])
        P = fa.RegParams(**lin)
        fn = fa.fa_affine_register if w == "affine" else fa.fa_rigid_register
        call = lambda: fn(fixed, moving, P, sync=False)["loss"]  # noqa
        cfg.update(lin, loss="lncc")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(None)
    clocks.start()
    launches0 = fa.fa_launch_count()
    last = None
    for k in range(args.steps):
        flush.zero_()
        e0[k].record(stream)
        last = call()
        e1[k].record(stream)
    torch.cuda.synchronize()
    launches = fa.fa_launch_count() - launches0
    clk = clocks.stop()
    total_ms = float(sum(a.elapsed_time(b) for a, b in zip(e0, e1)))
    value = vi * args.steps / (total_ms / 1e3)
    peak, peak_kind = measured_peak()
    achieved = VARIANT_BYTES[w] * vi * args.steps / (total_ms / 1e3) / 1e9
    cfg["l2"] = "flushed between steps (256 MiB write)"
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg,
            "roofline": {"bound": "hbm", "kernel": "whole_path", "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "bytes_per_voxel_iter": VARIANT_BYTES[w]},
            "clocks": clk, "gpu_launches": int(launches), "final_value": float(last),
            "e2e": None}
    if w == "microscopy":
        line["dtype"] = "f32"
        line["s_per_pair"] = total_ms / args.steps / 1e3
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = variant_oracle_sample(w, f, m, psi)
    print(json.dumps(line))
    return 0


def variant_oracle_sample(w, f, m, psi):
    """The oracle on one finest-level iteration of the workload (plus its final
    evaluation), as voxel-iterations per second."""
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    import oracle
    oracle.build()
    kw = dict(lr=WORKLOAD["lr"], sigma_grad=WORKLOAD["sigma_grad"],
              sigma_warp=WORKLOAD["sigma_warp"])
    t0 = time.perf_counter()
    if w == "symmetric":
        oracle.register_symmetric(f, m, [1], [1], inv_scales=(1,), inv_iters=(1,),
                                  window=WORKLOAD["window"], cc_eps=WORKLOAD["cc_eps"], **kw)
    elif w == "inverse":
        oracle.inverse(psi, [1], [1], **kw)
    elif w == "svf":
        oracle.register_svf(f, m, [1], [1], steps=SVF_STEPS, window=WORKLOAD["window"],
                            cc_eps=WORKLOAD["cc_eps"], **kw)
    elif w in ("mi", "use_jac"):
        oracle.register(f, m, [1], [1], loss="mi" if w == "mi" else "lncc",
                        use_jac=(w == "use_jac"), window=WORKLOAD["window"],
                        cc_eps=WORKLOAD["cc_eps"], **kw)
    elif w == "microscopy":
        oracle.register(f, m, [1], [1], window=MICROSCOPY["window"], cc_eps=WORKLOAD["cc_eps"],
                        **kw)
    elif w == "affine":
        oracle.affine_register(f, m, [1], [1], lr=3e-3, window=WORKLOAD["window"],
                               cc_eps=WORKLOAD["cc_eps"])
    else:
        oracle.rigid_register(f, m, [1], [1], lr=3e-3, window=WORKLOAD["window"],
                              cc_eps=WORKLOAD["cc_eps"])
    dt = time.perf_counter() - t0
    n = int(np.prod(f.shape))
    grid = "x".join(str(a) for a in f.shape)
    return {"value": n / dt, "unit": METRIC, "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle",
            "sample": f"1 finest-level iteration (scale 1, {grid}) of the same workload "
                      "plus the oracle's final evaluation"}


# --------------------------------------------- PyTorch-primitives comparison
def _torch_gauss_1d(sigma, dev):
    """Normalised Gaussian taps exp(-k^2 / 2 sigma^2), |k| <= ceil(3 sigma)."""
    import torch
    if sigma <= 0:
        return torch.ones(1, device=dev)
    r = int(np.ceil(3 * sigma))
    k = torch.arange(-r, r + 1, device=dev, dtype=torch.float64)
    w = torch.exp(-k * k / (2 * sigma * sigma))
    return (w / w.sum()).float()


def _torch_smooth(x, w):
    """Separable Gaussian of x [C, D, H, W] along z, y, x (zero outside)."""
    import torch.nn.functional as F
    c, r = x.shape[0], (w.numel() - 1) // 2
    if r == 0:
        return x
    y = x.unsqueeze(0)
    for axis in range(3):
        shape = [1, 1, 1]
        shape[axis] = w.numel()
        pad = [0, 0, 0]
        pad[axis] = r
        y = F.conv3d(y, w.view(1, 1, *shape).expand(c, 1, *shape).contiguous(), padding=pad,
                     groups=c)
    return y[0]


def _torch_grid(u):
    """Normalised sampling grid of x + u(x) (align-corners), [1, D, H, W, 3] in x, y, z order."""
    import torch
    _, D, H, W = u.shape
    z, y, x = torch.meshgrid(torch.arange(D, device=u.device), torch.arange(H, device=u.device),
                             torch.arange(W, device=u.device), indexing="ij")
    def norm(c, n):
        return c * (2.0 / max(n - 1, 1)) - 1.0
    gx = norm(x + u[2], W)
    gy = norm(y + u[1], H)
    gz = norm(z + u[0], D)
    return torch.stack([gx, gy, gz], dim=-1).unsqueeze(0)


def _torch_warp(img, u):
    """img [C, D, H, W] sampled at x + u(x), trilinear, zero outside."""
    import torch.nn.functional as F
    return F.grid_sample(img.unsqueeze(0), _torch_grid(u), mode="bilinear", padding_mode="zeros",
                         align_corners=True)[0]


def _torch_lncc(I, J, win, eps):
    """-mean cc of the box-window LNCC (window sums with zeros outside)."""
    import torch.nn.functional as F
    r = win // 2
    n = float(win ** 3)
    def box(v):
        return F.avg_pool3d(v[None, None], win, stride=1, padding=r, count_include_pad=True)[0, 0] * n
    sI, sJ, sII, sJJ, sIJ = box(I), box(J), box(I * I), box(J * J), box(I * J)
    cross = sIJ - sI * sJ / n
    varI = sII - sI * sI / n
    varJ = sJJ - sJ * sJ / n
    return -(cross * cross / (varI * varJ + eps)).mean()


def _torch_register(If0, Im0, scales, iters, lr, sg, sw, win, eps, b1=0.9, b2=0.999,
                    adam_eps=1e-8, c_lp=2.0):
    """Algorithm 1 (Jacobian-free direction) written with PyTorch primitives
    in the style of the paper's own implementation: grid_sample for the
    warps, pooling for the LNCC window sums, autograd for dL/du, separable
    convolutions for the Gaussians.  Returns (u, mean cc of the last level)."""
    import torch
    import torch.nn.functional as F
    dev = If0.device
    wg, ww = _torch_gauss_1d(sg, dev), _torch_gauss_1d(sw, dev)
    u = m = v = None
    prev = None
    t = 0
    for s, T in zip(scales, iters):
        dims = tuple(level_size(a, s) for a in If0.shape)
        def level(img):
            x = _torch_smooth(img[None], _torch_gauss_1d(0.5 * s, dev)) if s > 1 else img[None]
            if s > 1:
                x = F.interpolate(x[None], size=dims, mode="trilinear", align_corners=True)[0]
            return x[0]
        If, Im = level(If0), level(Im0)
        if u is None:
            u = torch.zeros((3,) + dims, device=dev)
            m = torch.zeros_like(u)
            v = torch.zeros_like(u)
        else:
            sa = torch.tensor([(f - 1) / (c - 1) if c > 1 and f > 1 else 1.0
                               for f, c in zip(dims, prev)], device=dev).view(3, 1, 1, 1)
            def up(x):
                return F.interpolate(x[None], size=dims, mode="trilinear", align_corners=True)[0]
            u, m, v = up(u) * sa, up(m) / sa, up(v) / (sa * sa)
        prev = dims
        for _ in range(T):
            t += 1
            u_ = u.detach().requires_grad_(True)
            L = _torch_lncc(If, _torch_warp(Im[None], u_)[0], win, eps)
            g, = torch.autograd.grad(L, u_)
            g = _torch_smooth(g, wg)
            m = b1 * m + (1 - b1) * g
            v = b2 * v + (1 - b2) * g * g
            d = (m / (1 - b1 ** t)) / (torch.sqrt(v / (1 - b2 ** t)) + adam_eps)
            delta = -(lr / (c_lp * d.norm(dim=0).max())) * d
            u = _torch_smooth(delta + _torch_warp(u, delta), ww)
    with torch.no_grad():
        L = _torch_lncc(If, _torch_warp(Im[None], u)[0], win, eps)
    return u, -float(L)


def run_torch_primitives(args):
    """The brain workload with the PyTorch-primitives form of the same
    iteration (a comparison point in the style of the paper's own code: its
    kernels are PyTorch's, not this library's), timed like the fused arm."""
    import torch
    from paper_2404_01249_gb300 import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    shape = WORKLOAD["shape"]
    f, m, _ = synth.voronoi_pair(shape=shape, seed=1000)
    If0, Im0 = torch.from_numpy(f).to(dev), torch.from_numpy(m).to(dev)
    kw = dict(scales=WORKLOAD["scales"], iters=WORKLOAD["iters"], lr=WORKLOAD["lr"],
              sg=WORKLOAD["sigma_grad"], sw=WORKLOAD["sigma_warp"], win=WORKLOAD["window"],
              eps=WORKLOAD["cc_eps"])
    for _ in range(args.warmup):
        _torch_register(If0, Im0, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        u, cc = _torch_register(If0, Im0, **kw)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    vi = voxel_iters(shape, WORKLOAD["scales"], WORKLOAD["iters"])
    print(json.dumps({"metric": METRIC, "value": vi / (ms / 1e3), "unit": METRIC,
                      "impl": "torch_primitives", "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                      "dtype": "f32", "data": "synthetic", "final_lncc": cc,
                      "config": {"workload": WORKLOAD["name"], "shape": list(shape),
                                 "scales": list(WORKLOAD["scales"]),
                                 "iters": list(WORKLOAD["iters"]),
                                 "form": "PyTorch primitives (grid_sample, avg_pool3d, "
                                         "conv3d, autograd); a comparison point, not this "
                                         "library's path"}}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fused", choices=["fused", "plain", "torch"],
                    help="fused or plain: this library's schedules; torch: the same iteration "
                         "written with PyTorch primitives (a comparison point)")
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default tile choices instead of fa_autotune's")
    ap.add_argument("--batched", type=int, default=0, metavar="P",
                    help="time fa_register_batched on P uneven pairs x 9 parameter sets instead")
    ap.add_argument("--concurrency", type=int, default=8,
                    help="streams of --batched's streams and plain schedules")
    ap.add_argument("--schedule", default="lockstep", choices=["lockstep", "streams", "plain"],
                    help="timed form of --batched")
    ap.add_argument("--field", default="f32", choices=["f32", "f16"],
                    help="storage of the displacement u between iterations (fused mode)")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16"],
                    help="--batched: storage of the images and Adam moments")
    ap.add_argument("--no-compare", action="store_true",
                    help="--batched: time only the chosen schedule (profiling runs)")
    ap.add_argument("--workload", default="brain",
                    choices=["brain", "symmetric", "inverse", "svf", "mi", "use_jac", "affine",
                             "rigid", "microscopy"],
                    help="one of the paper's other workloads on the brain-shaped pair, or "
                         "the microscopy-shaped pair at its full size")
    ap.add_argument("--scales", type=int, nargs="+", default=None,
                    help="override the pyramid scales (profiling runs; changes the workload)")
    ap.add_argument("--iters", type=int, nargs="+", default=None,
                    help="override the iterations per level (profiling runs)")
    args = ap.parse_args()
    if args.scales is not None or args.iters is not None:
        sc = tuple(args.scales or WORKLOAD["scales"])
        it = tuple(args.iters or WORKLOAD["iters"])
        if len(sc) != len(it):
            ap.error("--scales and --iters need the same length")
        WORKLOAD.update(scales=sc, iters=it,
                        name=WORKLOAD["name"] + "_scales" + "-".join(map(str, sc)) +
                        "_iters" + "-".join(map(str, it)))
    if args.impl == "reference":
        return run_reference(args)
    if args.batched:
        return run_batched(args)
    if args.workload != "brain":
        return run_variant(args)
    if args.mode == "torch":
        return run_torch_primitives(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
