#!/usr/bin/env python3
"""Benchmark of the fused two-component regularized colour-gradient step.

Metric: two-fluid MLUPS (million fluid-site updates per second, both components
advanced), with the HBM roofline fraction of the fused step kernel.

Default workload: the 3D step emulsifier, D3Q19, 768 x 128 x 32 box, FP32
deviation storage (the single large instance of the roofline measurement; its
two state buffers, 2 x 478 MB, are larger than the 129 MB L2, so no L2 flush is
needed between steps).  One bench step = one lattice update of the whole box.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lbcg|reference]
                       [--workload step_emulsifier|flow_focuser|droplet2d] [--precision f32dev|f32|f64|f16scaled]
For N > 1 (torchrun), every rank runs an independent replica (the path has no
exchange step on one box): value = all ranks' site updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1711_02003_gb300 import workloads as W  # noqa: E402

PREC = {"f64": 0, "f32": 1, "f32dev": 2, "f16scaled": 3}
DTYPE = {"f64": "f64", "f32": "f32", "f32dev": "f32", "f16scaled": "f32 (f16 storage)"}
ELEM = {"f64": 8, "f32": 4, "f32dev": 4, "f16scaled": 2}
OBS_EVERY = 100


def make_workload(name: str):
    if name == "step_emulsifier":
        pb = W.step_emulsifier()
        return pb, "3D step emulsifier D3Q19 768x128x32 (terrace 256x126x8, reservoir 512x126x30)", (384, 64, 16)
    if name == "flow_focuser":
        pb = W.cross_junction()
        return pb, "2D flow-focusing cross junction D2Q9 1024x192 (main channel 64, side inlets 64 at x=256)", (512, 96)
    if name == "droplet2d":
        pb = W.static_droplet(W.D2Q9, 4096, 512)
        return pb, "2D static droplet D2Q9 4096x4096 periodic, R=512", (2048, 2048)
    raise SystemExit(f"unknown workload {name}")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int = 0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def __enter__(self):
        def run():
            q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            while not self._stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                         timeout=5).stdout.strip()
                    if out:
                        self.samples.append([v.strip() for v in out.split(",")])
                except Exception:
                    pass
                self._stop.wait(0.1)
        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if len(s) > 2 + k and
                          s[2 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def reduce_max(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_sample(pb, budget_s: float = 12.0):
    """Time the FP64 oracle on the same workload: whole-box steps until budget_s."""
    import oracle
    s = oracle.Sim(pb)
    fluid = pb.fluid_sites()
    n = 0
    t0 = time.perf_counter()
    while True:
        s.step(1)
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": fluid * n / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{n} full-box step(s) of the same workload ({fluid} fluid sites), FP64, OpenMP over "
                      f"{oracle.threads()} host threads, {dt:.1f} s"}


def run_reference(args, world, rank):
    """The oracle timed as the reference arm (host cores)."""
    if rank != 0:
        return
    pb, desc, _ = make_workload(args.workload)
    import oracle
    s = oracle.Sim(pb)
    fluid = pb.fluid_sites()
    for _ in range(args.warmup):
        s.step(1)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    v = fluid * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": "two-fluid MLUPS", "value": v, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "precision": "f64 oracle (CPU)", "fluid_sites": fluid},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{args.steps} timed full-box steps after {args.warmup} warm-up"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="lbcg", choices=["lbcg", "reference"])
    ap.add_argument("--workload", default="step_emulsifier")
    ap.add_argument("--precision", default="f32dev", choices=list(PREC))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world, rank, local = dist_setup() if args.impl == "lbcg" else (int(os.environ.get("WORLD_SIZE", "1")),
                                                                    int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_1711_02003_gb300 import build as B
    from paper_1711_02003_gb300 import lbcg
    if not os.path.exists(B.LIB):
        B.build()
    lbcg.load()
    torch.cuda.set_device(local)
    pb, desc, centre = make_workload(args.workload)
    prec = PREC[args.precision]
    fluid = pb.fluid_sites()
    stream = torch.cuda.current_stream()

    # ---------------------------------------------------------------- device-resident run
    sim = lbcg.Simulation(pb, prec, stream=stream)
    sim.step(args.warmup)
    sim.observables(centre, allow_diverged=True)
    torch.cuda.synchronize()
    n_obs = (args.steps + OBS_EVERY - 1) // OBS_EVERY
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sim.set_kernel_timing(True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        done = 0
        while done < args.steps:
            k = min(OBS_EVERY, args.steps - done)
            sim.step(k)
            done += k
            sim.observables(centre, allow_diverged=True)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    kms, klaunch = sim.kernel_time()
    sim.set_kernel_timing(False)
    ms_max = reduce_max(ms, world)
    value = world * fluid * args.steps / (ms_max * 1e-3) / 1e6
    obs = sim.observables(centre, allow_diverged=True)
    port_launch = 1 if pb.ports else 0
    launches = args.steps * (1 + port_launch) + n_obs * 4

    # ---------------------------------------------------------------- roofline of the step kernel
    elem = ELEM[args.precision]
    bytes_per_site = 2 * 2 * pb.q * elem          # read 2Q + write 2Q populations
    k_avg_s = kms / klaunch * 1e-3
    achieved = bytes_per_site * fluid / k_avg_s / 1e9
    peak, peak_kind = peaks()

    # ---------------------------------------------------------------- end to end through host buffers
    n = pb.nsites
    h_rr = torch.from_numpy(np.ascontiguousarray(pb.rho_r, np.float64)).pin_memory()
    h_rb = torch.from_numpy(np.ascontiguousarray(pb.rho_b, np.float64)).pin_memory()
    o_rr = torch.empty(n, dtype=torch.float64).pin_memory()
    o_rb = torch.empty(n, dtype=torch.float64).pin_memory()
    o_u = torch.empty(pb.dim * n, dtype=torch.float64).pin_memory()
    L = lbcg.load()
    import ctypes as C
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbcg._check("lbcg_init_fields", L.lbcg_init_fields(sim._h, C.c_void_p(h_rr.data_ptr()),
                                                       C.c_void_p(h_rb.data_ptr()), None))
    done = 0
    while done < args.steps:
        k = min(OBS_EVERY, args.steps - done)
        sim.step(k)
        done += k
        sim.observables(centre, allow_diverged=True)
    lbcg._check("lbcg_get_fields", L.lbcg_get_fields(sim._h, C.c_void_p(o_rr.data_ptr()),
                                                     C.c_void_p(o_rb.data_ptr()), C.c_void_p(o_u.data_ptr())))
    e2e_s = time.perf_counter() - t0
    e2e_s = reduce_max(e2e_s, world)
    e2e_value = world * fluid * args.steps / e2e_s / 1e6
    h2d = 2 * n * 8
    d2h = (2 + pb.dim) * n * 8
    barrier(world)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(pb, args.cpu_budget)
    clocks = clk.summary()
    line = {
        "metric": "two-fluid MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": desc, "lattice": "D2Q9" if pb.lattice == 0 else "D3Q19",
                   "precision": args.precision, "fluid_sites": fluid, "box_sites": n,
                   "steps_per_observable": OBS_EVERY, "l2": "state (2 buffers) larger than L2, no flush"
                   if 2 * sim.state_bytes > 4 * 129e6 else "state fits in L2 (not a roofline instance)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "fused step", "bytes_per_site": bytes_per_site,
                     "kernel_ms_avg": k_avg_s * 1e3, "peak_source": peak_kind},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps, "h2d_bytes_total": h2d, "d2h_bytes_total": d2h,
                "note": "one job: upload initial densities, K steps with observables every 100, read back fields"},
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "observables": {"mass_r": obs["mass_r"], "mass_b": obs["mass_b"], "umax": obs["umax"],
                        "nonfinite": obs["nonfinite"]},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
