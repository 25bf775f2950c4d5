"""Continuous-batching server for simulation requests.

Requests (lattice, geometry, Capillary number, viscosity ratio, step count) arrive over
time.  A request is admitted as soon as (a) it has arrived, (b) its state fits in the
HBM budget next to the resident requests and (c) its lattice's batch has a free slot;
admission is first-come first-served.  Admitted requests keep their populations
resident on the device and advance together in the batch of their lattice (one
persistent fused kernel per lattice per step, replayed from a captured CUDA graph), so
work from requests that arrived at different times overlaps on the GPU.  Finished
requests are read back (observables), their memory is freed and waiting requests take
their place.  The server reports time-to-result (finish - arrival) percentiles and the
aggregate throughput.  A request withdrawn by its client (cancel_at) leaves the queue or is
evicted from the device; with health checks on, a resident instance whose density went
non-finite is evicted early; a finished one is reported diverged.  Neither disturbs the
other requests.

The scheduling logic talks to an Engine; :class:`LbcgEngine` runs the CUDA library, and
tests substitute a host-only engine.
"""
from __future__ import annotations

import dataclasses
import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads as W


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the run
    problem: W.Problem
    steps: int
    centre: tuple = None
    cancel_at: float = None   # the client withdraws the request at this time (None: never)


@dataclass
class Result:
    rid: int
    lattice: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    fluid_sites: int
    observables: dict = field(default_factory=dict)
    status: str = "done"      # "done", "cancelled" (withdrawn), "diverged" (evicted)

    @property
    def time_to_result(self) -> float:
        return self.finished - self.arrival


def make_requests(n: int, rate: float = 20.0, seed: int = 0, steps_scale: float = 1.0) -> list:
    """n requests of the mixed serving workload with Poisson arrivals of mean `rate`/s."""
    arrivals = W.poisson_arrivals(n, rate, seed)
    out = []
    for k in range(n):
        spec = W.random_request(seed * 1000003 + k)
        pb = W.serving_problem(spec)
        steps = max(1, int(round(spec["steps"] * steps_scale)))
        centre = (pb.nx / 2, pb.ny / 2, pb.nz / 2)
        out.append(Request(k, float(arrivals[k]), pb, steps, centre))
    return out


class Engine:
    """What the server needs from a backend."""

    def state_bytes(self, req: Request) -> int:
        raise NotImplementedError

    def free_slots(self, lattice: int) -> int:
        raise NotImplementedError

    def admit(self, req: Request):
        """Create the instance on the device and queue it; returns a handle."""
        raise NotImplementedError

    def advance(self, steps: int):
        """Advance every resident instance by up to `steps` steps (asynchronous)."""
        raise NotImplementedError

    def finished(self) -> list:
        """Handles of the instances that completed (waits for outstanding work)."""
        raise NotImplementedError

    def retire(self, handle) -> dict:
        """Read back the observables of a finished instance and free its memory."""
        raise NotImplementedError

    def resident(self) -> int:
        raise NotImplementedError

    def evict(self, handle) -> None:
        """Remove an unfinished instance and free its memory (cancellation, divergence)."""
        raise NotImplementedError

    def diverged(self, handle) -> bool:
        """Health check of a resident instance (only called when the server asks for checks)."""
        return False


class LbcgEngine(Engine):
    """The CUDA library: one lbcg batch per lattice on a shared stream."""

    def __init__(self, precision: int = 2, max_slots: int = 64, stream=None, shapes: dict | None = None):
        """shapes: optional launch shape per lattice ({W.D2Q9: {...}, W.D3Q19: {...}}, fields of
        lbcg_batch_shape), e.g. from autotune.autotune_batch."""
        import torch

        from . import lbcg
        self.lb = lbcg
        lbcg.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.precision = precision
        shapes = shapes or {}
        self.batches = {lat: lbcg.Batch(lat, precision, max_slots, stream=self.stream, shape=shapes.get(lat))
                        for lat in (W.D2Q9, W.D3Q19)}
        self.handles = {}

    def state_bytes(self, req: Request) -> int:
        # two population buffers + the per-site link table
        return 2 * self.lb.state_bytes(req.problem, self.precision) + 4 * req.problem.nsites

    def free_slots(self, lattice: int) -> int:
        b = self.batches[lattice]
        return b.max_instances - b.active

    def admit(self, req: Request):
        sim = self.lb.Simulation(req.problem, self.precision, stream=self.stream)
        b = self.batches[req.problem.lattice]
        slot = b.add(sim, req.steps)
        h = (req.problem.lattice, slot)
        self.handles[h] = (sim, req)
        return h

    def advance(self, steps: int):
        for b in self.batches.values():
            if b.active:
                b.step(steps)

    def finished(self) -> list:
        out = []
        for lat, b in self.batches.items():
            if b.active:
                out += [(lat, s) for s in b.poll()]
        return out

    def retire(self, handle) -> dict:
        sim, req = self.handles.pop(handle)
        obs = sim.observables(req.centre, allow_diverged=True)
        self.batches[handle[0]].remove(handle[1])
        sim.close()
        return obs

    def resident(self) -> int:
        return len(self.handles)

    def evict(self, handle) -> None:
        sim, _ = self.handles.pop(handle)
        self.batches[handle[0]].remove(handle[1])
        sim.close()

    def diverged(self, handle) -> bool:
        sim, req = self.handles[handle]
        return sim.observables(req.centre, allow_diverged=True)["nonfinite"] > 0


class Server:
    """Continuous batching under an HBM budget (see the module docstring)."""

    def __init__(self, engine: Engine, hbm_budget: float = 150e9, chunk: int = 100, health_every: int = 0):
        self.engine = engine
        self.budget = float(hbm_budget)
        self.chunk = int(chunk)
        self.health_every = int(health_every)  # chunks between health checks of the residents (0: none)
        self.used = 0.0
        self.peak_used = 0.0
        self.peak_resident = 0

    def run(self, requests: list, realtime: bool = True, clock=time.perf_counter) -> list:
        queue = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in queue:
            need = self.engine.state_bytes(r)
            if need > self.budget:
                raise ValueError(f"request {r.rid} needs {need} bytes, more than the whole budget")
        t0 = clock()
        vclock = 0.0  # simulated clock when not realtime

        def now():
            return clock() - t0 if realtime else vclock

        live = {}
        results = []
        nchunks = 0

        def drop(h, status):
            r, need, t_adm = live.pop(h)
            self.engine.evict(h)
            self.used -= need
            results.append(Result(r.rid, r.problem.lattice, r.arrival, t_adm, now(), r.steps,
                                  r.problem.fluid_sites(), {}, status))

        while queue or live:
            # withdrawn requests: dropped from the queue, evicted from the device
            t = now()
            for r in [r for r in queue if r.cancel_at is not None and r.cancel_at <= t]:
                queue.remove(r)
                results.append(Result(r.rid, r.problem.lattice, r.arrival, -1.0, t, r.steps,
                                      r.problem.fluid_sites(), {}, "cancelled"))
            for h in [h for h, (r, _, _) in live.items() if r.cancel_at is not None and r.cancel_at <= t]:
                drop(h, "cancelled")
            if self.health_every and nchunks and nchunks % self.health_every == 0:
                for h in [h for h in live if self.engine.diverged(h)]:
                    drop(h, "diverged")
            if not queue and not live:
                break
            # the resident requests advance asynchronously; the host admits meanwhile, so
            # instance set-up (allocation, geometry tables, initial state) overlaps GPU work
            advanced = bool(live)
            if advanced:
                self.engine.advance(self.chunk)
                nchunks += 1
                if not realtime:
                    vclock += 1e-3
            # admission: arrived, fits the budget, free slot (first come, first served)
            t = now()
            while queue and queue[0].arrival <= t:
                r = queue[0]
                need = self.engine.state_bytes(r)
                if self.used + need > self.budget or self.engine.free_slots(r.problem.lattice) == 0:
                    break
                h = self.engine.admit(r)
                live[h] = (r, need, now())
                self.used += need
                self.peak_used = max(self.peak_used, self.used)
                queue.pop(0)
            self.peak_resident = max(self.peak_resident, len(live))
            if not live:
                if queue:
                    if realtime:
                        time.sleep(max(0.0, queue[0].arrival - now()))
                    else:
                        vclock = max(vclock, queue[0].arrival)
                continue
            if not advanced:
                continue
            for h in self.engine.finished():
                r, need, t_adm = live.pop(h)
                obs = self.engine.retire(h)
                self.used -= need
                status = "diverged" if obs.get("nonfinite", 0) > 0 else "done"
                results.append(Result(r.rid, r.problem.lattice, r.arrival, t_adm, now(), r.steps,
                                      r.problem.fluid_sites(), obs, status))
        return sorted(results, key=lambda x: x.rid)


def summary(results: list) -> dict:
    """p50/p99 time-to-result and aggregate MLUPS (fluid-site updates / makespan) over the
    completed requests; withdrawn and diverged requests are counted apart."""
    done = [r for r in results if r.status == "done"]
    if not done:
        return {"requests": 0, "cancelled": len(results), "diverged": 0} if results else {}
    ttr = np.array([r.time_to_result for r in done])
    start = min(r.arrival for r in results)
    end = max(r.finished for r in done)
    work = sum(r.fluid_sites * r.steps for r in done)
    return {"requests": len(done), "cancelled": sum(r.status == "cancelled" for r in results),
            "diverged": sum(r.status == "diverged" for r in results),
            "p50_s": float(np.percentile(ttr, 50)), "p99_s": float(np.percentile(ttr, 99)),
            "mean_s": float(ttr.mean()), "makespan_s": end - start, "site_updates": int(work),
            "aggregate_mlups": work / max(end - start, 1e-12) / 1e6}


def run_one_at_a_time(requests: list, precision: int = 0, clock=time.perf_counter) -> list:
    """Baseline: first-come first-served, one request at a time on the GPU (no batching)."""
    import torch

    from . import lbcg
    lbcg.load()
    queue = sorted(requests, key=lambda r: (r.arrival, r.rid))
    t0 = clock()
    results = []
    for r in queue:
        t = clock() - t0
        if t < r.arrival:
            time.sleep(r.arrival - t)
        t_adm = clock() - t0
        sim = lbcg.Simulation(r.problem, precision)
        sim.step(r.steps)
        obs = sim.observables(r.centre, allow_diverged=True)
        torch.cuda.synchronize()
        sim.close()
        results.append(Result(r.rid, r.problem.lattice, r.arrival, t_adm, clock() - t0, r.steps,
                              r.problem.fluid_sites(), obs))
    return results
