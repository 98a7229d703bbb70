#!/usr/bin/env python3
"""Throughput benchmark of the two-species multi-range LB step on GB300.

Workload (default): the rho0 sweep at the paper's resolution -- five periodic
512 x 512 lattices, FP32, rho0 in {0.55, 0.65, 0.70, 0.75, 0.83}, the Fig. 2
caption couplings, Psi = rho0 (1 - exp(-rho/rho0)), seeded init (seed 1).
One bench step = one LB time step of all five lattices (5 x 512^2 two-species
site updates).  Metric: MLUPS (million two-species site updates per second).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lbinputs  # noqa: E402

BYTES_PER_SITE = {"fp64": 288, "fp32": 144, "fp16": 72, "bf16": 72}
# the sources that define the step kernel's code
KERNEL_SRCS = [os.path.join(ROOT, "paper_0807_4471_gb300", "csrc", f)
               for f in ("lb_kernels.cu", "lb_layout.cuh", "lb_internal.h")]


def kernel_hash() -> str:
    """sha256 (16 hex digits) of the step kernel's sources with comments and
    runs of blank space removed: it changes with the code, not the prose."""
    h = hashlib.sha256()
    for path in KERNEL_SRCS:
        with open(path) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel: str, precision: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; None otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(f"{kernel}:{precision}:{workload}")
    if not e or e.get("kernel_sha") != kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.th.join(timeout=2)

    def summary(self):
        mhz, maxmhz, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                maxmhz.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(maxmhz),
                "reasons": sorted(reasons), "samples": len(mhz)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(dist, value: float, device=None) -> float:
    """The slowest rank's time (the bench's clock for N replicas)."""
    import torch
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Weak scaling: every rank runs the full workload; value = all ranks'
    units / the slowest rank's time."""
    return units_per_rank * world / seconds


def time_steps(torch, lats, steps: int):
    """CUDA-event time of `steps` bench steps on the lattices' stream."""
    stream = lats[0].stream
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        for g in lats:
            g.step(1)
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def cpu_oracle_sample(nx: int, ny: int, rho0: float, steps: int, seed: int):
    import oracle as O
    c = lbinputs.CAPTION
    P = O.make_params(nx, ny, Ga=c["Ga"], Gr=c["Gr"], GX=c["GX"], rho0=rho0, psi_form=1)
    f = O.init_seeded(P, seed)
    t0 = time.perf_counter()
    O.run(P, f, steps)
    dt = time.perf_counter() - t0
    return nx * ny * steps / dt / 1e6, dt


def _oracle_worker(args):
    """One process of the parallel oracle baseline: `warm` untimed steps, then
    `steps` timed steps of one sweep lattice (spawned: no CUDA state)."""
    nx, ny, rho0, warm, steps, seed = args
    import oracle as O
    c = lbinputs.CAPTION
    P = O.make_params(nx, ny, Ga=c["Ga"], Gr=c["Gr"], GX=c["GX"], rho0=rho0, psi_form=1)
    f = O.init_seeded(P, seed)
    O.run(P, f, warm)
    t0 = time.perf_counter()
    O.run(P, f, steps, t0=warm)
    return time.perf_counter() - t0


def cpu_oracle_parallel(nx: int, ny: int, rho0s, warm: int, steps: int, seed: int):
    """The oracle, as it stands, on several host cores at once: one process
    per lattice (rho0s), each stepping its own lattice.  Returns (aggregate
    MLUPS = all updates / the slowest process's time, that time, processes)."""
    import multiprocessing as mp
    import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    jobs = [(nx, ny, r0, warm, steps, seed) for r0 in rho0s]
    with ctx.Pool(len(jobs)) as pool:
        dts = pool.map(_oracle_worker, jobs)
    dt = max(dts)
    return nx * ny * steps * len(jobs) / dt / 1e6, dt, len(jobs)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    """The reference arm: the FP64 oracle on the same workload as the GPU arm
    -- one bench step is one LB step of every lattice of the rho0 sweep --
    with one process per lattice on the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cfg = lbinputs.CFG_SWEEP
    nx, ny = args.nx, args.ny
    rho0s = list(cfg["rho0s"][:args.lattices])
    value, dt, nproc = cpu_oracle_parallel(nx, ny, rho0s, args.warmup, args.steps, cfg["seed"])
    sample = (f"all {len(rho0s)} lattices of the rho0 sweep ({nx}x{ny}, rho0 {rho0s}), "
              f"{args.steps} timed steps after {args.warmup} warm-up steps, FP64 oracle, one "
              f"process per lattice on {nproc} of the {host_cores()} host cores")
    line = {
        "impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"rho0 sweep, {len(rho0s)} x {nx}x{ny} periodic lattices; a bench "
                               "step is one LB step of all of them", "nx": nx, "ny": ny,
                   "lattices": len(rho0s), "rho0": rho0s},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": nproc, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def peak_lattice(torch, lb, precision: str, n: int, steps: int, tile_rows: int = 0):
    """MLUPS and algorithmic GB/s of one large periodic lattice (inputs >> L2)
    with the given step-kernel tile height (0: the library default)."""
    p = lb.make_params(n, n, precision, psi_form=lb.LB_PSI_RHO0, tile_rows=tile_rows)
    g = lb.Lattice(p).init_seeded(lbinputs.CFG_PEAK["seed"])
    g.step(3)
    torch.cuda.synchronize()
    dt = time_steps(torch, [g], steps)
    g.sync()
    g.close()
    mlups = n * n * steps / dt / 1e6
    return mlups, mlups * 1e6 * BYTES_PER_SITE[precision] / 1e9


def batched_mix(torch, lb, steps: int, precision: str = "fp16"):
    """The batched workload: 64 lattices (sizes from {128, 256, 512, 1024}^2,
    rho0 in [0.55, 0.83], half Couette), FP16 offsets (or `precision`), one
    pool launch per step, every lattice run for `steps` steps.  Aggregate
    MLUPS over the whole run, CUDA events on the pool's stream around it:
    the partition tuning on the first steps (real steps of the jobs) and the
    CUDA-graph capture are inside."""
    jobs = lbinputs.sample_batch()
    stream = torch.cuda.Stream()
    shared = lb.make_params(128, 128, precision, psi_form=lb.LB_PSI_RHO0)
    params = []
    for j in jobs:
        params.append(lb.make_params(j["nx"], j["ny"], precision, psi_form=lb.LB_PSI_RHO0,
                                     rho0=j["rho0"], boundary=j["boundary"],
                                     u_wall=lbinputs.wall_speed(j["shear_rate"], j["ny"]),
                                     init_shear=j["boundary"]))
    budget = sum(lb.Pool.footprint(p) for p in params) + (64 << 20)
    with lb.Pool(shared, budget, max_jobs=len(params), stream=stream) as pool:
        ids = [pool.admit(p, j["seed"], steps) for p, j in zip(params, jobs)]
        stream.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        while pool.run(steps):
            pass
        ev1.record(stream)
        ev1.synchronize()
        dt = ev0.elapsed_time(ev1) / 1e3
        for i in ids:
            pool.stress(i)   # raises on a latched device error
        sites = sum(p.nx * p.ny for p in params)
        return {"MLUPS": sites * steps / dt / 1e6, "lattices": len(params), "sites": sites,
                "steps": steps, "seconds": dt, "segment": pool.segment,
                "tile_rows": pool.tile_rows,
                "ms_per_step": dt / steps * 1e3,
                "GB_per_s_alg": sites * steps * BYTES_PER_SITE[precision] / dt / 1e9}


def serving(torch, lb, njobs: int, step_scale: float, load: float, capacity_mlups: float,
            precision: str = "fp16"):
    """The served workload: the first `njobs` requests of the seeded arrival
    stream (square lattices 64..2048, rho0 in [0.55, 0.83], shear rate 0 or
    one of the 8 Couette rates), step counts scaled by `step_scale`, Poisson
    arrivals at `load` x `capacity_mlups`.  Jobs are served by the
    continuous-batching server over a lattice pool (FP16 offsets, or
    `precision`)."""
    from paper_0807_4471_gb300.serve import Server, job_params, percentile
    specs = lbinputs.sample_serving()[:njobs]
    for sp in specs:
        sp["steps"] = max(10, int(round(sp["steps"] * step_scale)))
    work = np.mean([sp["nx"] * sp["ny"] * sp["steps"] for sp in specs])
    gap = work / (load * capacity_mlups * 1e6)          # mean inter-arrival time (s)
    stream = [(sp["arrival"] * gap, sp) for sp in specs]
    make = job_params(lb, dict(psi_form=lb.LB_PSI_RHO0), precision)
    cuda_stream = torch.cuda.Stream()
    budget = 48 << 30
    pool = lb.Pool(make(dict(nx=64, ny=64)), budget, max_jobs=1024, stream=cuda_stream)
    srv = Server(pool, make, quantum=100)
    t0 = time.perf_counter()
    jobs = srv.replay(stream)
    makespan = time.perf_counter() - t0
    pool.close()
    lat = [j.latency for j in jobs if j.error is None]
    return {"jobs": len(jobs), "failed": sum(1 for j in jobs if j.error), "p50_s": percentile(lat, 50),
            "p99_s": percentile(lat, 99), "MLUPS": srv.stats.site_updates / makespan / 1e6,
            "makespan_s": makespan, "step_scale": step_scale, "load": load,
            "mean_interarrival_s": gap, "quantum": srv.quantum, "precision": precision,
            "refused_nomem": srv.stats.refused_nomem}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 5000; the reference arm, a CPU oracle: 200)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=list(BYTES_PER_SITE))
    ap.add_argument("--nx", type=int, default=lbinputs.CFG_SWEEP["nx"])
    ap.add_argument("--ny", type=int, default=lbinputs.CFG_SWEEP["ny"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-peak", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--tune-steps", type=int, default=600,
                    help="untimed set-up steps on which the pool tunes its work partition")
    ap.add_argument("--settle-s", type=float, default=0.5,
                    help="untimed seconds of steps before the warm-up (clock record under load)")
    ap.add_argument("--batch-steps", type=int, default=lbinputs.CFG_BATCH_STEPS,
                    help="steps of every lattice of the 64-lattice batch")
    ap.add_argument("--boundary", default="periodic", choices=["periodic", "couette"],
                    help="the sweep lattices' boundary (couette: moving walls, shear rate 1e-4)")
    ap.add_argument("--tile-rows", type=int, default=0,
                    help="fix the step kernel's tile height (8 or 16; 0: autotuned with the partition)")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-scale", type=float, default=0.1,
                    help="factor on the served jobs' step counts")
    ap.add_argument("--lattices", type=int, default=len(lbinputs.CFG_SWEEP["rho0s"]),
                    help="number of sweep lattices stepped per bench step (profiling runs)")
    ap.add_argument("--kernel-hash", action="store_true",
                    help="print the step kernel's source hash (as the traffic record keys it) and exit")
    args = ap.parse_args()
    if args.kernel_hash:
        print(kernel_hash())
        return 0
    if args.steps is None:
        args.steps = 200 if args.impl == "reference" else 5000
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_0807_4471_gb300 as lb
    from paper_0807_4471_gb300 import build as _b

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    _b.build()
    lb.load()

    cfg = lbinputs.CFG_SWEEP
    nx, ny, prec = args.nx, args.ny, args.precision
    rho0s = list(cfg["rho0s"][:args.lattices])
    stream = torch.cuda.Stream()
    wall = {} if args.boundary == "periodic" else dict(
        boundary=lb.LB_COUETTE, u_wall=lbinputs.wall_speed(1e-4, ny), init_shear=1)
    shared = lb.make_params(nx, ny, prec, psi_form=lb.LB_PSI_RHO0)
    budget = sum(lb.Pool.footprint(lb.make_params(nx, ny, prec, rho0=r0, psi_form=lb.LB_PSI_RHO0,
                                                  **wall)) for r0 in rho0s) + (64 << 20)
    pool = lb.Pool(shared, budget, max_jobs=len(rho0s), stream=stream)
    if args.tile_rows:
        pool.set_tile_rows(args.tile_rows)
    # members run until released: the untimed set-up, warm-up, timed and
    # end-to-end steps all come out of one long schedule
    jobs = [pool.admit(lb.make_params(nx, ny, prec, rho0=r0, psi_form=lb.LB_PSI_RHO0, **wall),
                       cfg["seed"], 1 << 40) for r0 in rho0s]

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # The clock record spans the set-up, the warm-up and the timed steps, so
    # that a short timed region still has samples taken under load.
    with ClockSampler(local) as clk:
        # Set-up, untimed: the pool's autotuner times its candidate
        # partitions on the first steps of the member set (real steps), then
        # the launch of the chosen partition is captured into a CUDA graph.
        pool.run(args.tune_steps)
        pool.prepare()
        stream.synchronize()
        # untimed steps until the sampler has seen the GPU under load
        settle, t_set = 0, time.perf_counter()
        while time.perf_counter() - t_set < args.settle_s:
            pool.run(1024)
            stream.synchronize()
            settle += 1024
        pool.run(args.warmup)
        barrier()
        ev0.record(stream)
        pool.run(args.steps)
        ev1.record(stream)
        ev1.synchronize()
    dt = ev0.elapsed_time(ev1) / 1e3
    barrier()
    for j in jobs:
        pool.stress(j)   # raises on a latched device error
    dt = max_over_ranks(dist, dt, device="cuda")
    sites = nx * ny * len(rho0s)
    value = replica_throughput(sites * args.steps, ws, dt) / 1e6
    launches = args.steps          # one persistent launch per step for all lattices
    avg_launch = dt / launches
    hbm_peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_SITE[prec] * sites / avg_launch / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                "traffic": ncu_traffic("k_step", prec, f"{len(rho0s)}x{nx}x{ny}"),
                "traffic_source": "profiles/traffic.json (ncu, taken on this kernel source)",
                "bytes_per_launch_alg": BYTES_PER_SITE[prec] * sites,
                "kernel": f"k_step<{prec}> (all {len(rho0s)} lattices per launch, "
                          f"{pool.tile_rows}-row tiles)",
                "avg_launch_us": avg_launch * 1e6, "segment": pool.segment,
                "tile_rows": pool.tile_rows}
    pool_segment, pool_rows = pool.segment, pool.tile_rows

    # End to end through the public API with host buffers: restart the same
    # pool members from FP64 fields in pinned host memory (host -> device),
    # take the steps, read rho_A and rho_B back (device -> host); the member
    # set, its tuned partition and its graph are the ones timed above.
    e2e = None
    if not args.no_e2e:
        def pinned(shape):
            return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        host = []
        for k in range(len(jobs)):
            u = lbinputs.uniforms(100 + k, (2, ny, nx))
            r0 = rho0s[k]
            ra, rb = pinned((ny, nx)), pinned((ny, nx))
            ra[:] = r0 * (1 + 0.03 * (2 * u[0] - 1))
            rb[:] = r0 * (1 + 0.03 * (2 * u[1] - 1))
            host.append((ra, rb))
        outA = [pinned((ny, nx)) for _ in jobs]
        outB = [pinned((ny, nx)) for _ in jobs]
        e_steps = args.steps
        barrier()
        t0 = time.perf_counter()
        for (ra, rb), j in zip(host, jobs):
            pool.init_fields(j, ra, rb)
        pool.run(e_steps)
        for j, a, b in zip(jobs, outA, outB):
            lb.lb_pool_fields(pool.h, j, a, b, None, None)
        e_dt = time.perf_counter() - t0
        e_dt = max_over_ranks(dist, e_dt, device="cuda")
        h2d = sum(a.nbytes + b.nbytes for a, b in host)
        d2h = sum(a.nbytes + b.nbytes for a, b in zip(outA, outB))
        e2e = {"value": replica_throughput(sites * e_steps, ws, e_dt) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / e_steps, "d2h_bytes_per_step": d2h / e_steps,
               "note": "lattice pool through the C ABI: lb_pool_init_fields of every member from "
                       "pinned host FP64 fields, the steps, lb_pool_fields of rho_A and rho_B to "
                       "pinned host memory; bytes amortised per step"}
    pool.close()

    extra = {}
    if rank == 0 and not args.no_peak:
        # FP32 and the two 16-bit offset formats (BF16: the same kernel code as
        # FP16 with the other 16-bit type)
        for p in ("fp32", "fp16", "bf16"):
            by_rows = {}
            for rows in (8, 16):
                mlups, gbs = peak_lattice(torch, lb, p, lbinputs.CFG_PEAK["nx"], 50, rows)
                by_rows[rows] = {"MLUPS": mlups, "GB_per_s_alg": gbs, "frac_hbm": gbs / hbm_peak}
            best = max(by_rows, key=lambda r: by_rows[r]["MLUPS"])
            n = lbinputs.CFG_PEAK["nx"]
            gbs = by_rows[best]["GB_per_s_alg"]
            # the HBM-roofline claim of the step kernel: inputs far larger than L2
            roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": gbs / hbm_peak, "peak_kind": peak_kind,
                    "bytes_per_launch_alg": BYTES_PER_SITE[p] * n * n,
                    "traffic": ncu_traffic("k_step", p, f"1x{n}x{n}") if best == 16 else None,
                    "traffic_source": "profiles/traffic.json (ncu, 16-row tiles, this kernel source)"}
            extra[f"peak_{p}_4096"] = dict(by_rows[best], tile_rows=best, roofline=roof,
                                           by_tile_rows={str(r): v for r, v in by_rows.items()})
        extra["batched_64_fp16"] = batched_mix(torch, lb, args.batch_steps)
        extra["batched_64_fp32"] = batched_mix(torch, lb, args.batch_steps, "fp32")
        if not args.no_serve:
            # the same arrival stream (rate set by the FP16 batched capacity) for both
            cap = extra["batched_64_fp16"]["MLUPS"]
            extra["serving"] = serving(torch, lb, args.serve_jobs, args.serve_scale, 0.8, cap)
            extra["serving_fp32"] = serving(torch, lb, args.serve_jobs, args.serve_scale, 0.8,
                                            cap, "fp32")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        steps_cpu = 60
        mlups, cdt = cpu_oracle_sample(nx, ny, 0.70, steps_cpu, cfg["seed"])
        ncores = host_cores()
        lat = [rho0s[k % len(rho0s)] for k in range(ncores)]
        par, pdt, nproc = cpu_oracle_parallel(nx, ny, lat, 0, 30, cfg["seed"])
        cpu = {"value": par, "unit": "MLUPS", "cores": nproc, "kind": "oracle",
               "sample": f"{nproc} processes, one per host core ({ncores}), each stepping one "
                         f"{nx}x{ny} lattice of the sweep (rho0 cycling over {rho0s}) 30 steps, "
                         f"{pdt:.1f} s; aggregate over the slowest process's time; FP64 oracle "
                         "as it stands",
               "single_core": {"value": mlups, "unit": "MLUPS", "cores": 1,
                               "sample": f"one {nx}x{ny} lattice (rho0 0.70), {steps_cpu} steps, "
                                         f"{cdt:.1f} s, one thread"}}

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f16-offset storage, f32 math",
                      "bf16": "bf16-offset storage, f32 math"}[prec],
            "data": "synthetic",
            "config": {"workload": f"rho0 sweep, {len(rho0s)} x {nx}x{ny} {args.boundary} lattices, "
                                   f"{prec} storage; a bench step is one LB step of all of them, "
                                   "one persistent launch (lattice pool, CUDA-graph replay)",
                       "nx": nx, "ny": ny, "lattices": len(rho0s),
                       "rho0": list(cfg["rho0s"]), "couplings": "Fig. 2 caption",
                       "l2": "inputs larger than L2, no flush: the lattices' two population "
                             "buffers (194 MB for 5 x 512^2 at FP32) alternate every step, each "
                             "step reading the previous step's output; when one buffer of all "
                             "lattices fits in L2 (97 MB here) the kernel stores it evict-last, "
                             "so part of it is still in L2 when the next step reads it, as in "
                             "any run of consecutive steps",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "setup": f"untimed before the warm-up: {args.tune_steps} steps of "
                                "partition autotuning, CUDA-graph capture of the chosen launch, "
                                f"{settle} steps while the clock sampler starts",
                       "partition": pool_segment, "tile_rows": pool_rows},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk.summary(), "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
