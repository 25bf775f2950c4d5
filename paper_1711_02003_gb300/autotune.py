"""Launch-shape autotuner for the fused step.

For one problem and storage precision it times the fused step kernel (CUDA events
around every launch, lbcg_set_kernel_timing) for each candidate launch shape on a
scratch instance, and returns the fastest.  All candidates compute the same update
(bit-identical within one kernel variant, rounding-level across variants), so tuning
never changes results beyond rounding.

Candidates:
  D2Q9 : rows per warp strip in {2, 4, 8, 16, 32, 64} x variant {6 moment march (regularized),
         1 plain march} (short strips give small boxes enough warps)
  D3Q19: warps per block along y in {4, 6, 8} x z-planes per block in {4, 8, 16} x
         variant; regularized collision {7, 6 moment march (shared-memory / register
         moments), 5 re-read}, plus 12 and 16 warps per block for variant 7, the moment march
         with neighbour-only plane barriers (variant 9; 6 or 8 warps) and the TMA-staged march
         (variant 8; 6 or 8 warps, 8 or 16 planes) for 4-byte storage; BGK {5, 1, 2}; FP64
         regularized {6, 7, 2, 9 (6 or 8 warps)}, BGK {2, 1}

autotune_batch times the batched kernels' launch shapes (work-item cut, resident blocks per
SM, steps per captured graph) on a set of instances, such as a sample of the serving mix.

Run as a program it prints the candidate table of one named workload, in launch order
(each candidate: `warm` untimed then `steps` timed launches of its step kernel):

    python -m paper_1711_02003_gb300.autotune --workload step_emulsifier --precision f32dev
"""
from __future__ import annotations

import argparse
import itertools
import json

from . import lbcg

_CACHE = {}


def candidates(lattice: int, precision: int, collision: int = 0) -> list:
    if lattice == lbcg.LBCG_D2Q9:
        vs = (6, 1) if collision == 0 else (1,)  # moment march (regularized only), plain march
        return [dict(rows=r, block_rows=0, variant=v) for v, r in itertools.product(vs, (2, 4, 8, 16, 32, 64))]
    f64 = precision == lbcg.LBCG_FP64
    if collision == 0:  # regularized
        variants = [6, 7, 2] if f64 else [7, 6, 5]
    else:
        variants = [2, 1] if f64 else [5, 1, 2]
    out = [dict(rows=r, block_rows=b, variant=v) for v, b, r in itertools.product(variants, (4, 6, 8), (4, 8, 16))]
    if collision == 0:
        out += [dict(rows=r, block_rows=b, variant=9) for b, r in itertools.product((6, 8), (4, 8, 16))]
    if 7 in variants:
        out += [dict(rows=r, block_rows=b, variant=7) for b, r in itertools.product((12, 16), (4, 8))]
        if lbcg.ELEM_BYTES[precision] == 4:  # TMA-staged march (runs as 7 where it does not apply)
            out += [dict(rows=r, block_rows=b, variant=8) for b, r in itertools.product((6, 8), (8, 16))]
    return out


def kernel_ms(sim, steps: int = 30, warm: int = 5) -> float:
    import torch
    sim.step(warm)
    torch.cuda.synchronize()
    sim.set_kernel_timing(True)
    sim.step(steps)
    ms, n = sim.kernel_time()
    sim.set_kernel_timing(False)
    return ms / max(n, 1)


def autotune(pb, precision: int, steps: int = 30, cands: list | None = None, cache: bool = True) -> dict:
    """Fastest launch shape for problem `pb`: {'rows', 'block_rows', 'variant', 'ms', 'table'}."""
    key = (pb.lattice, pb.nx, pb.ny, pb.nz, precision, pb.collision, pb.fluid_sites())
    if cache and key in _CACHE:
        return _CACHE[key]
    table = []
    for c in (cands or candidates(pb.lattice, precision, pb.collision)):
        sim = lbcg.Simulation(pb, precision, **c)
        table.append(dict(c, ms=kernel_ms(sim, steps)))
        sim.close()
        del sim
    best = min(table, key=lambda t: t["ms"])
    out = dict(best, table=table)
    if cache:
        _CACHE[key] = out
    return out


def batch_candidates(lattice: int) -> list:
    """Batch launch shapes tried by autotune_batch (graph_steps is tuned after them)."""
    if lattice == lbcg.LBCG_D2Q9:
        return [dict(rows=r, strips_per_item=s, blocks_per_sm=b)
                for r, s, b in itertools.product((8, 16, 32), (2, 4, 8), (0, 2))]
    return [dict(rows=r, block_rows=w, blocks_per_sm=b) for w, r, b in itertools.product((4, 6, 8), (4, 8, 16), (0, 2))]


def autotune_batch(problems: list, precision: int, steps: int = 64, cands: list | None = None,
                   graph_steps=(16, 32, 64)) -> dict:
    """Fastest batch launch shape for a set of instances of one lattice (e.g. a sample of the
    serving mix): all of them go into one batch, each candidate shape times `steps` steps of
    the whole batch (CUDA events on the batch's stream, after a warm-up that captures the
    graph), then the steps per graph are tuned for the best shape.  Returns {'shape', 'mlups',
    'table'}; aggregate MLUPS = fluid sites of all instances x steps / time."""
    import torch
    lattice = problems[0].lattice
    stream = torch.cuda.Stream()
    batch = lbcg.Batch(lattice, precision, len(problems), stream=stream)
    sims = [lbcg.Simulation(pb, precision, stream=stream) for pb in problems]
    for sim in sims:
        batch.add(sim, 1 << 40)
    fluid = sum(pb.fluid_sites() for pb in problems)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(shape):
        batch.set_shape(**shape)
        gs = batch.shape["graph_steps"]
        batch.step(2 * gs)
        stream.synchronize()
        e0.record(stream)
        batch.step(steps)
        e1.record(stream)
        stream.synchronize()
        return fluid * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6

    table = [dict(c, mlups=timed(c)) for c in (cands or batch_candidates(lattice))]
    best = max(table, key=lambda t: t["mlups"])
    base = {k: v for k, v in best.items() if k != "mlups"}
    for g in graph_steps:
        table.append(dict(base, graph_steps=g, mlups=timed(dict(base, graph_steps=g))))
    best = max(table, key=lambda t: t["mlups"])
    batch.set_shape(**{k: v for k, v in best.items() if k != "mlups"})
    out = {"shape": batch.shape, "mlups": best["mlups"], "instances": len(problems), "steps": steps, "table": table}
    for slot in list(batch.sims):
        batch.remove(slot)
    for sim in sims:
        sim.close()
    batch.close()
    return out


PRECISIONS = {"f64": 0, "f32": 1, "f32dev": 2, "f16scaled": 3}


def main(argv=None):
    from . import workloads as W
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="step_emulsifier", choices=W.NAMED)
    ap.add_argument("--precision", default="f32dev", choices=list(PRECISIONS))
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warm", type=int, default=5)
    args = ap.parse_args(argv)
    lbcg.load()
    pb, desc, _ = W.named(args.workload)
    prec = PRECISIONS[args.precision]
    table = []
    for c in candidates(pb.lattice, prec, pb.collision):
        sim = lbcg.Simulation(pb, prec, **c)
        table.append(dict(c, ms=kernel_ms(sim, args.steps, args.warm)))
        sim.close()
        del sim
    best = min(table, key=lambda t: t["ms"])
    print(json.dumps({"workload": desc, "precision": args.precision, "warm": args.warm, "steps": args.steps,
                      "fluid_sites": pb.fluid_sites(), "best": best, "table": table}))


if __name__ == "__main__":
    main()
