#!/usr/bin/env python3
"""Benchmark of the fused two-component regularized colour-gradient step.

Metric: two-fluid MLUPS (million fluid-site updates per second, both components
advanced), with the HBM roofline fraction of the fused step kernel.

Default workload: the 3D step emulsifier, D3Q19, 768 x 128 x 32 box, FP32
deviation storage (the single large instance of the roofline measurement; its
two state buffers, 2 x 478 MB, are larger than the 129 MB L2, so no L2 flush is
needed between steps).  One bench step = one lattice update of the whole box.

Timed region: K steps in chunks of 100 (three replays of the library's 32-step CUDA
graph plus four individual launches; both graphs captured before the region) with the
observables after each chunk.  Each chunk of steps, and nothing else, is bracketed by CUDA
events on the launching stream; the summed chunk time over the steps is the kernel time of
the roofline figure (an upper bound: it includes the gaps between consecutive kernels).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lbcg|reference]
                       [--workload step_emulsifier|flow_focuser|droplet2d|droplet3d] [--precision f32dev|f32|f64|f16scaled]
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
    try:
        return W.named(name)
    except ValueError as e:
        raise SystemExit(str(e))


def recorded(kind: str, workload: str, precision: str, launch: dict):
    """A per-launch ncu figure of the step kernel (kind "traffic": DRAM bytes read + written;
    kind "flops": executed FP64 / FP32 flops) from the records committed under profiles/
    for this workload, precision and launch shape, when the step-kernel sources are
    unchanged since (their digest is part of the record); else None."""
    from paper_1711_02003_gb300 import build as B
    digest = B.step_kernel_digest()
    want = {"workload": workload, "precision": precision, "variant": str(launch["variant"]),
            "block_rows": str(launch["block_rows"]), "rows": str(launch["rows"]), "digest": digest}
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None, digest
    for name in sorted(os.listdir(pdir)):
        if not name.endswith((".md", ".txt")):
            continue
        with open(os.path.join(pdir, name)) as f:
            for line in f:
                line = line.strip().strip("`")
                if not line.startswith(kind + "-record:"):
                    continue
                kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
                if all(kv.get(k) == v for k, v in want.items()):
                    return kv, digest
    return None, digest


def roofline_alu(alu: dict, traffic, k_avg_s: float, hbm_achieved: float, hbm_peak: float, bytes_per_site: int,
                 fluid: int, digest: str) -> dict:
    """FP64 runs are bound by the FP64 rate: the roofline is the ALU one (TFLOP/s), with the
    HBM figures beside it."""
    ach = None if alu["achieved_gflops"] is None else alu["achieved_gflops"] / 1e3
    return {"bound": "alu", "achieved": ach, "peak": alu["fma_peak_gflops"] / 1e3, "unit": "TFLOP/s",
            "frac": alu["frac"], "traffic": traffic, "kernel": "fused step (FP64)",
            "flops_per_launch": alu["flops_per_launch"], "kernel_ms_avg": k_avg_s * 1e3,
            "peak_source": "lbcg_fma_peak (FP64 FMA chains, measured in this run)",
            "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
                    "bytes_per_site": bytes_per_site, "algorithmic_bytes": bytes_per_site * fluid},
            "kernel_digest": digest}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """SM clock and throttle reasons sampled by one streaming nvidia-smi (-lms 50) over the
    GPU-loaded part of the run; samples read between mark_start() and mark_end() belong to
    the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0, period_ms: int = 50):
        self.index = index
        self.period_ms = period_ms
        self.samples = []          # (host time, fields)
        self.window = None
        self._proc = None
        self._t = None

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                           "--format=csv,noheader,nounits", f"-lms={self.period_ms}"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self._proc = None
            return self

        def run():
            for line in self._proc.stdout:
                vals = [v.strip() for v in line.strip().split(",")]
                if len(vals) >= 2:
                    self.samples.append((time.perf_counter(), vals))
        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()
        return self

    def mark_start(self):
        self.window = [time.perf_counter(), None]

    def mark_end(self):
        if self.window:
            self.window[1] = time.perf_counter()

    def __exit__(self, *a):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()
        if self._t:
            self._t.join(timeout=5)

    def summary(self):
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        allv = [v for _, v in self.samples]
        timed = [v for t, v in self.samples if self.window and self.window[1] and self.window[0] <= t <= self.window[1]]
        use = timed if timed else allv
        sm = [x for x in (num(v[0]) for v in use) if x is not None]
        mx = [x for x in (num(v[1]) for v in allv) if x is not None]
        reasons = sorted({names[k] for v in allv for k in range(4) if len(v) > 2 + k and v[2 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(allv), "samples_timed": len(timed),
                "window": "timed region" if timed else "GPU-loaded run (warm-up, timed region, end-to-end phase)",
                "period_ms": self.period_ms}


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


def reduce_max(v: float, world: int, device: str = "cuda") -> float:
    """Max over ranks (the slowest replica sets the job's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(units_per_rank: float, world: int, ms_local: float, device: str = "cuda") -> tuple:
    """Whole-job throughput of `world` replicas: all ranks' site updates over the max-over-ranks
    time.  Returns (MLUPS, max ms)."""
    ms_max = reduce_max(ms_local, world, device)
    return world * units_per_rank / (ms_max * 1e-3) / 1e6, ms_max


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_sample(pb, budget_s: float = 12.0):
    """Time the FP64 oracle on the same workload: whole-box steps until budget_s.
    Returns the cpu_baseline record and the oracle (advanced by the timed steps)."""
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
    rec = {"value": fluid * n / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
           "sample": f"{n} full-box step(s) of the same workload ({fluid} fluid sites), FP64, OpenMP over "
                     f"{oracle.threads()} host threads, {dt:.1f} s"}
    return rec, s


def cpu_suite() -> dict:
    """The FP64 oracle timed on the host cores, single-threaded and over all threads (the
    results are bit-identical across thread counts): C1 in full, the C3 box at R = 16 for a
    bounded number of steps."""
    import platform

    import oracle
    allt = oracle.threads()
    cases = [("C1 static droplet D2Q9 64x64 R=16", W.static_droplet(W.D2Q9, 64, 16), 2000, 2000),
             ("C3 static droplet D3Q19 128^3 R=16", W.static_droplet(W.D3Q19, 128, 16), 50, 4)]
    rows = []
    for name, pb, n_all, n_one in cases:
        for nt, n in ((allt, n_all), (1, n_one)):
            oracle.set_threads(nt)
            sim = oracle.Sim(pb)
            t0 = time.perf_counter()
            sim.step(n)
            dt = time.perf_counter() - t0
            rows.append({"workload": name, "threads": nt, "steps": n, "seconds": dt,
                         "MLUPS": pb.fluid_sites() * n / dt / 1e6})
    oracle.set_threads(allt)
    return {"cpu_suite": rows, "host": {"machine": platform.machine(), "cpus": os.cpu_count(), "model": cpu_model()},
            "kind": "oracle"}


def cpu_model() -> str:
    """The host CPU's model line from /proc/cpuinfo (x86: model name; Arm: implementer and part)."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read().splitlines()
    except OSError:
        return "unknown"
    for key in ("model name", "Model name"):
        for line in info:
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    impl = next((ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU implementer")), "?")
    part = next((ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU part")), "?")
    return f"implementer {impl} part {part}"


def error_vs_oracle(sim, osim) -> dict:
    """Max-norm relative error of the GPU fields against the FP64 oracle after the same steps."""
    gr, gb, gu = sim.fields()
    orr, ob, ou = osim.fields()

    def rel(a, b):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    return {"steps": int(osim.step_count), "rho_r": rel(gr, orr), "rho_b": rel(gb, ob), "u": rel(gu, ou),
            "u_abs": float(np.abs(gu - ou).max())}


def serving_sample(n_requests: int, steps_scale: float, baseline_n: int, rate: float = 20.0,
                   slots: int = 64) -> dict:
    """Continuous-batching serving of the mixed request workload (FP32-dev batches under a
    150 GB HBM budget) and the one-at-a-time FP64 baseline on the first requests."""
    from paper_1711_02003_gb300 import autotune, serve
    reqs = serve.make_requests(n_requests, rate=rate, seed=0, steps_scale=steps_scale)
    # batch launch shapes tuned (untimed) on the first 16 requests of each lattice of the mix
    tuned = {}
    for lat in (W.D2Q9, W.D3Q19):
        sample = [r.problem for r in serve.make_requests(96, rate=rate, seed=1) if r.problem.lattice == lat][:16]
        t = autotune.autotune_batch(sample, PREC["f32dev"])
        tuned[lat] = {"shape": t["shape"], "mlups": t["mlups"], "instances": t["instances"],
                      "candidates": len(t["table"])}
    eng = serve.LbcgEngine(precision=PREC["f32dev"], max_slots=slots,
                           shapes={lat: t["shape"] for lat, t in tuned.items()})
    srv = serve.Server(eng, hbm_budget=150e9, chunk=100)
    res = srv.run(reqs, realtime=True)
    out = {"requests": n_requests, "arrival_rate_per_s": rate, "steps_scale": steps_scale, "hbm_budget_gb": 150,
           "slots_per_lattice": slots,
           "batch_shapes": {"D2Q9": tuned[W.D2Q9], "D3Q19": tuned[W.D3Q19]},
           "precision": "f32dev", "peak_resident": srv.peak_resident, "peak_hbm_gb": srv.peak_used / 1e9}
    out.update({k: v for k, v in serve.summary(res).items()})
    if baseline_n:
        base = serve.run_one_at_a_time(reqs[:baseline_n], precision=PREC["f64"])
        bs = serve.summary(base)
        out["baseline_one_at_a_time_f64"] = {"requests": baseline_n, "p50_s": bs["p50_s"], "p99_s": bs["p99_s"],
                                             "aggregate_mlups": bs["aggregate_mlups"]}
    return out


def accuracy_gate(err: dict, pb) -> dict:
    """FP32 accuracy gate against the FP64 oracle (max-norm relative, every field after the CPU
    sample's steps).  u is gated with the densities; in a resting droplet u is the spurious
    current alone and the 1e-5 relative gate on it is not met (stated below)."""
    dens = err["rho_r"] <= 1e-5 and err["rho_b"] <= 1e-5
    u_ok = err["u"] <= 1e-5
    gate = {"fields_rel_tol": 1e-5, "steps": err["steps"], "rho_passed": bool(dens), "u_passed": bool(u_ok),
            "passed": bool(dens and u_ok),
            "note": "FP32 gate of rho_R, rho_B and u against the FP64 oracle (max-norm relative); FP16-scaled "
                    "storage is reported and fails it by design"}
    if not pb.ports:
        gate["u_at_rest"] = ("not met at rest: u of a resting droplet is the spurious current alone (about 5e-5 in "
                             "2D, 1e-6 in 3D) and FP32 rounding leaves about 2e-9 absolute error, i.e. 4.5e-5 (2D) "
                             "and 2e-4 (3D) relative after 1000 steps; the tests gate u at rest at 1e-8 absolute")
    return gate


def prime_graphs(sim):
    """Capture the library's step graphs (one per starting buffer) before a timed region: 66
    untimed steps that end on the starting buffer they began on."""
    for n in (32, 1, 32, 1):
        sim.step(n)


def _kernel_timed(sim, steps: int, stream):
    """Average duration (s) of the step kernel over `steps` consecutive steps (CUDA events on the
    library's stream around the steps only, launched as the library launches them: graphs of 32
    steps, no events between launches, so the average includes the gaps between kernels) and the
    wall time (ms) of those steps on the stream."""
    import torch
    sim.step(3)
    prime_graphs(sim)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return ms / (steps * sim.grid["kernels_per_step"]) * 1e-3, ms


def fp64_sample(lbcg, pb, stream, fluid: int, workload: str, steps: int = 20) -> dict:
    """The same workload with FP64 storage and arithmetic (library default launch shape), the
    plain FP64 GPU path the FP32 path is compared with: kernel and whole-step MLUPS over
    `steps` steps, and its roofline, which is the FP64 ALU rate (executed flops from the
    committed ncu record of this kernel source and shape; HBM beside it)."""
    sim = lbcg.Simulation(pb, PREC["f64"], stream=stream)
    k_avg, whole_ms = _kernel_timed(sim, steps, stream)
    launch = sim.launch
    rec_f, digest = recorded("flops", workload, "f64", launch)
    flops = int(rec_f["fp64_flops"]) if rec_f else None
    fma = lbcg.fma_peak(0, stream)
    peak, peak_kind = peaks()
    bps = 2 * 2 * pb.q * 8
    sim.close()
    return {"precision": "f64", "steps": steps, "launch": launch, "kernel_ms_avg": k_avg * 1e3,
            "mlups_kernel": fluid / k_avg / 1e6, "mlups_whole": fluid * steps / (whole_ms * 1e-3) / 1e6,
            "roofline": {"bound": "alu", "unit": "TFLOP/s", "peak": fma / 1e3,
                         "achieved": None if flops is None else flops / k_avg / 1e12,
                         "frac": None if flops is None else flops / k_avg / 1e9 / fma,
                         "flops_per_launch": flops, "kernel_digest": digest,
                         "peak_source": "lbcg_fma_peak (FP64 FMA chains, measured in this run)",
                         "hbm": {"achieved": bps * fluid / k_avg / 1e9, "peak": peak, "unit": "GB/s",
                                 "frac": bps * fluid / k_avg / 1e9 / peak, "bytes_per_site": bps,
                                 "peak_source": peak_kind}}}


def roofline_2d_sample(lbcg, stream, steps: int = 20) -> dict:
    """The 4096^2 D2Q9 droplet (state far larger than L2), FP32-dev, library default launch
    shape: the 2D roofline instance, kernel time over `steps` consecutive launches."""
    pb, desc, _ = W.named("droplet2d")
    sim = lbcg.Simulation(pb, PREC["f32dev"], stream=stream)
    k_avg, whole_ms = _kernel_timed(sim, steps, stream)
    fluid = pb.fluid_sites()
    bps = 2 * 2 * pb.q * 4
    peak, peak_kind = peaks()
    out = {"workload": desc, "precision": "f32dev", "steps": steps, "launch": sim.launch,
           "kernel_ms_avg": k_avg * 1e3, "mlups_kernel": fluid / k_avg / 1e6,
           "mlups_whole": fluid * steps / (whole_ms * 1e-3) / 1e6,
           "roofline": {"bound": "hbm", "achieved": bps * fluid / k_avg / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": bps * fluid / k_avg / 1e9 / peak, "bytes_per_site": bps,
                        "algorithmic_bytes": bps * fluid, "peak_source": peak_kind}}
    sim.close()
    return out


def run_reference(args, world, rank, budget_s: float = 120.0):
    """The oracle timed as the reference arm on the host cores: full-box steps of the same
    workload, at most K timed steps and at most budget_s seconds (a bounded sample)."""
    if rank != 0:
        return
    pb, desc, _ = make_workload(args.workload)
    import oracle
    s = oracle.Sim(pb)
    fluid = pb.fluid_sites()
    warm = min(args.warmup, 3)
    s.step(warm)
    n = 0
    t0 = time.perf_counter()
    while n < args.steps:
        s.step(1)
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    v = fluid * n / dt / 1e6
    line = {"impl": "reference", "metric": "two-fluid MLUPS", "value": v, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "precision": "f64 oracle (CPU)", "fluid_sites": fluid},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{n} timed full-box steps (of {args.steps} requested, {budget_s:.0f} s cap) "
                                       f"after {warm} warm-up, FP64, OpenMP over {oracle.threads()} host threads"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="lbcg", choices=["lbcg", "reference"])
    ap.add_argument("--workload", default="step_emulsifier")
    ap.add_argument("--precision", default="f32dev", choices=list(PREC))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-suite", action="store_true",
                    help="only time the FP64 oracle on C1 / C3 (1 and all host threads) and print that line")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-autotune", action="store_true", help="library default launch shape")
    ap.add_argument("--launch", default=None, help="rows,block_rows,variant: this launch shape (no autotuning)")
    ap.add_argument("--serving-requests", type=int, default=64, help="0 disables the serving sample")
    ap.add_argument("--serving-steps-scale", type=float, default=0.25)
    ap.add_argument("--serving-baseline", type=int, default=6)
    ap.add_argument("--serving-slots", type=int, default=64, help="batch slots per lattice")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the FP64 sample and the 2D roofline instance")
    ap.add_argument("--serving-only", action="store_true",
                    help="only run the serving workload (--serving-requests, --serving-steps-scale) and print it")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world, rank, local = dist_setup() if args.impl == "lbcg" else (int(os.environ.get("WORLD_SIZE", "1")),
                                                                    int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.cpu_suite:
        if rank == 0:
            print(json.dumps(cpu_suite()), flush=True)
        return
    if args.serving_only:
        if rank == 0:
            import torch
            from paper_1711_02003_gb300 import lbcg
            lbcg.load()
            torch.cuda.set_device(local)
            t0 = time.perf_counter()
            out = serving_sample(args.serving_requests, args.serving_steps_scale, args.serving_baseline,
                                 slots=args.serving_slots)
            print(json.dumps({"serving": out, "wall_s": time.perf_counter() - t0}), flush=True)
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

    # ---------------------------------------------------------------- launch shape (untimed)
    shape = {}
    tuned = None
    if args.launch:
        r_, b_, v_ = (int(t) for t in args.launch.split(","))
        shape = {"rows": r_, "block_rows": b_, "variant": v_}
    elif not args.no_autotune:
        from paper_1711_02003_gb300 import autotune
        tuned = autotune.autotune(pb, prec)
        shape = {k: tuned[k] for k in ("rows", "block_rows", "variant")}

    # ---------------------------------------------------------------- device-resident run
    clk = ClockSampler(local).__enter__()
    sim = lbcg.Simulation(pb, prec, stream=stream, **shape)
    sim.step(args.warmup)
    prime_graphs(sim)
    sim.observables(centre, allow_diverged=True)
    torch.cuda.synchronize()
    n_obs = (args.steps + OBS_EVERY - 1) // OBS_EVERY
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # step-kernel time: events on the library's stream around each chunk of steps only (the
    # observables run between chunks), nothing between the chunk's launches
    chunk_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_obs)]
    barrier(world)
    torch.cuda.synchronize()
    clk.mark_start()
    ev0.record(stream)
    done = 0
    for c0, c1 in chunk_ev:
        k = min(OBS_EVERY, args.steps - done)
        c0.record(stream)
        sim.step(k)
        c1.record(stream)
        done += k
        sim.observables(centre, allow_diverged=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk.mark_end()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    kms = sum(c0.elapsed_time(c1) for c0, c1 in chunk_ev)
    klaunch = args.steps * sim.grid["kernels_per_step"]
    value, ms_max = aggregate_mlups(fluid * args.steps, world, ms)
    obs = sim.observables(centre, allow_diverged=True)
    grid = sim.grid
    launches = args.steps * grid["kernels_per_step"] + n_obs * 4

    # ---------------------------------------------------------------- roofline of the step kernel
    elem = ELEM[args.precision]
    bytes_per_site = 2 * 2 * pb.q * elem          # read 2Q + write 2Q populations
    k_avg_s = kms / klaunch * 1e-3
    achieved = bytes_per_site * fluid / k_avg_s / 1e9
    peak, peak_kind = peaks()
    eff_launch = sim.launch
    rec_t, digest = recorded("traffic", args.workload, args.precision, eff_launch)
    traffic = int(rec_t["dram_bytes"]) if rec_t else None
    rec_f, _ = recorded("flops", args.workload, args.precision, eff_launch)
    # FMA rate of the compute precision on this device (untimed with respect to the run)
    fma_gflops = lbcg.fma_peak(0 if args.precision == "f64" else 1, stream)
    flops_launch = None
    if rec_f:
        flops_launch = int(rec_f["fp64_flops"] if args.precision == "f64" else rec_f["fp32_flops"])
    alu = {"fma_peak_gflops": fma_gflops, "precision": "fp64" if args.precision == "f64" else "fp32",
           "flops_per_launch": flops_launch,
           "flops_per_fluid_site": None if flops_launch is None else flops_launch / fluid,
           "achieved_gflops": None if flops_launch is None else flops_launch / k_avg_s / 1e9,
           "frac": None if flops_launch is None else flops_launch / k_avg_s / 1e9 / fma_gflops,
           "source": "executed flops (2 FMA + ADD + MUL, ncu record in profiles/, psi-ring recomputation "
                     "included) / kernel time; peak = lbcg_fma_peak measured now"}

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

    # ---------------------------------------------------------------- FP64 path and 2D roofline (rank 0)
    fp64 = None
    r2d = None
    if rank == 0 and args.extras and args.precision != "f64":
        fp64 = fp64_sample(lbcg, pb, stream, fluid, args.workload)
        if args.workload != "droplet2d":
            r2d = roofline_2d_sample(lbcg, stream)
    clk.__exit__()

    if rank != 0:
        return
    cpu = None
    err = None
    if world == 1 and not args.no_cpu_baseline:
        cpu, osim = cpu_oracle_sample(pb, args.cpu_budget)
        sim.init_fields(pb.rho_r, pb.rho_b, pb.u)
        sim.step(osim.step_count)
        err = error_vs_oracle(sim, osim)
        if fp64 is not None:
            s64 = lbcg.Simulation(pb, PREC["f64"], stream=stream)
            s64.step(osim.step_count)
            fp64["error_vs_f64_oracle"] = error_vs_oracle(s64, osim)
            s64.close()
    serving = None
    if world == 1 and args.serving_requests > 0:
        serving = serving_sample(args.serving_requests, args.serving_steps_scale, args.serving_baseline)
    clocks = clk.summary()
    line = {
        "metric": "two-fluid MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": desc, "lattice": "D2Q9" if pb.lattice == 0 else "D3Q19",
                   "precision": args.precision, "fluid_sites": fluid, "box_sites": n,
                   "steps_per_observable": OBS_EVERY, "l2": "state (2 buffers) larger than L2, no flush"
                   if 2 * sim.state_bytes > 4 * 129e6 else "state fits in L2 (not a roofline instance)",
                   "parallelism": f"replicas x{world}",
                   "launch": dict(eff_launch, **grid, tuned=tuned is not None,
                                  tuned_ms=None if tuned is None else tuned["ms"],
                                  candidates=None if tuned is None else len(tuned["table"]))},
        "roofline": roofline_alu(alu, traffic, k_avg_s, achieved, peak, bytes_per_site, fluid, digest)
        if args.precision == "f64" else
                    {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_source": "ncu record in profiles/ (dram__bytes_read.sum + "
                     "dram__bytes_write.sum, one launch)" if traffic else "no ncu record for this kernel source and "
                     "launch shape", "algorithmic_bytes": bytes_per_site * fluid, "kernel_digest": digest,
                     "kernel": "fused step", "bytes_per_site": bytes_per_site,
                     "kernel_ms_avg": k_avg_s * 1e3, "kernel_timing": "CUDA events around each chunk of "
                     "consecutive step launches (observables outside), summed / steps", "peak_source": peak_kind},
        "alu": alu,
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps, "h2d_bytes_total": h2d, "d2h_bytes_total": d2h,
                "note": "one job: upload initial densities, K steps with observables every 100, read back fields"},
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "error_vs_f64_oracle": err,
        "accuracy_gate": None if err is None else accuracy_gate(err, pb),
        "fp64": fp64,
        "roofline_2d": r2d,
        "serving": serving,
        "observables": {"mass_r": obs["mass_r"], "mass_b": obs["mass_b"], "umax": obs["umax"],
                        "nonfinite": obs["nonfinite"]},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
