"""The bounds-checked debug build (compiled with -DLBCG_CHECK_BOUNDS).

Every population, link-word and psi-ring index of the step kernels is checked before the
access; an index outside its array would be skipped and reported through the context's
status word (LBCG_ERR_BOUNDS from lbcg_synchronize).  This test builds that library, loads
it in a separate process (one library per process), runs the small, ragged and walled/ported
parity cases in every step-kernel variant and checks that the status word stays zero and the
results still match the FP64 oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, ROOT)
import oracle
from paper_1711_02003_gb300 import lbcg, workloads as W
lbcg.load(LIB)
assert lbcg._lib.lbcg_bounds_checked() == 1
cases = [
    (W.static_droplet(W.D3Q19, 33, 1, ny=3, nz=4), 30, [{}]),
    (W.static_droplet(W.D3Q19, 5, 1, ny=5, nz=1), 30, [{}]),
    (W.static_droplet(W.D3Q19, 24, 6.5, ny=20, nz=18, centre=(11.5, 9.5, 8.5)), 40,
     [{}, dict(variant=5), dict(variant=7, block_rows=12, rows=5), dict(variant=1, block_rows=4, rows=3)]),
    (W.step_emulsifier(nx=64, ny=30, nz=10, terrace_len=20, terrace_h=4, u_in=0.01, fill_x=10), 60,
     [{}, dict(variant=5), dict(variant=7, block_rows=6, rows=3), dict(variant=8, block_rows=8, rows=4),
      dict(variant=2, block_rows=5, rows=7), dict(variant=9, block_rows=4, rows=5)]),
    (W.static_droplet(W.D2Q9, 61, 9, ny=37, tau_r=1.7, tau_b=0.8), 50, [{}, dict(variant=1, rows=3)]),
    (W.cross_junction(nx=130, channel_w=16, side_x=40, side_len=12, fill_x=30), 60, [{}, dict(variant=1, rows=5)]),
]
for pb, n, shapes in cases:
    o = oracle.Sim(pb)
    o.step(n)
    orr, orb, _ = o.fields()
    for shape in shapes:
        for prec, tol in ((lbcg.LBCG_FP64, 1e-11), (lbcg.LBCG_FP32_DEV, 1e-5)):
            g = lbcg.Simulation(pb, prec, **shape)
            g.step(n)
            g.synchronize()  # raises LbcgError (LBCG_ERR_BOUNDS) if any guard fired
            rr, rb, _ = g.fields()
            err = max(np.abs(rr - orr).max(), np.abs(rb - orb).max())
            assert err <= tol, (pb.name, shape, prec, err)
print("bounds-checked build: all cases clean")
"""


def test_bounds_checked_build_runs_clean():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02003_gb300 import build
    lib = build.build(checked=True)
    code = f"ROOT = {ROOT!r}\nLIB = {lib!r}\n" + CHILD
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "all cases clean" in r.stdout
