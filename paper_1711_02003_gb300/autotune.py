"""Launch-shape autotuner for the fused step.

For one problem and storage precision it times the fused step kernel (CUDA events
around every launch, lbcg_set_kernel_timing) for each candidate launch shape on a
scratch instance, and returns the fastest.  All candidates compute the same update
(bit-identical within one kernel variant, rounding-level across variants), so tuning
never changes results beyond rounding.

Candidates:
  D2Q9 : rows per warp strip in {8, 16, 32, 64} x variant {0 plain march, 3 pipelined}
  D3Q19: warps per block along y in {4, 6, 8} x z-planes per block in {4, 8, 16} x
         variant {5 re-read at three blocks per SM, 1 registers, 2 re-read,
         4 asynchronous copies (4-byte storage only)}; FP64 tries {2, 1}
"""
from __future__ import annotations

import itertools

from . import lbcg

_CACHE = {}


def candidates(lattice: int, precision: int) -> list:
    if lattice == lbcg.LBCG_D2Q9:
        return [dict(rows=r, block_rows=0, variant=v) for v, r in itertools.product((0, 3), (8, 16, 32, 64))]
    variants = [5, 1, 2] + ([4] if lbcg.ELEM_BYTES[precision] == 4 else [])
    if precision == lbcg.LBCG_FP64:
        variants = [2, 1]
    return [dict(rows=r, block_rows=b, variant=v) for v, b, r in itertools.product(variants, (4, 6, 8), (4, 8, 16))]


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
    key = (pb.lattice, pb.nx, pb.ny, pb.nz, precision, pb.fluid_sites())
    if cache and key in _CACHE:
        return _CACHE[key]
    table = []
    for c in (cands or candidates(pb.lattice, precision)):
        sim = lbcg.Simulation(pb, precision, **c)
        table.append(dict(c, ms=kernel_ms(sim, steps)))
        sim.close()
        del sim
    best = min(table, key=lambda t: t["ms"])
    out = dict(best, table=table)
    if cache:
        _CACHE[key] = out
    return out
