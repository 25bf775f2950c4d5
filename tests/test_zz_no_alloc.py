"""lbcg_observables_noalloc: the allocation-free observables entry point.

Some callers cannot allocate device memory (code recording a CUDA graph by stream
capture, plug-ins whose host application owns every allocation, loops that forbid
allocation after start-up).  This entry point needs no context and keeps its
reduction scratch in a file-scope device array; these checks call it through the C
ABI and compare it with lbcg_observables on the same state, twice in a row, so the
shared scratch carries nothing from one call into the next."""
import ctypes as C

import numpy as np
import pytest

from paper_1711_02003_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    ("droplet D2Q9 64^2", lambda: W.static_droplet(W.D2Q9, 64, 16), (32, 32, 0), False),
    ("step emulsifier D3Q19 70x20x12", lambda: W.step_emulsifier(nx=70, ny=20, nz=12, terrace_len=24,
                                                                   terrace_h=4, u_in=0.01, fill_x=12),
     (35, 10, 6), True),
]


@pytest.fixture(scope="module")
def lb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02003_gb300 import build
    build.build()
    from paper_1711_02003_gb300 import lbcg
    lbcg.load()
    return lbcg


def _noalloc(lb, sim, mask_dev, centre, r_in=-1.0, r_out=-1.0):
    L = lb.load()
    out = lb.lbcg_obs()
    c = (C.c_double * 3)(*[float(v) for v in centre])
    st = L.lbcg_observables_noalloc(C.byref(sim._p), C.c_void_p(sim._a.data_ptr()),
                                    None if mask_dev is None else C.c_void_p(mask_dev.data_ptr()), c,
                                    float(r_in), float(r_out), C.c_void_p(sim.stream.cuda_stream), C.byref(out))
    assert st == 0, L.lbcg_last_error().decode()
    return out


@pytest.mark.parametrize("name,make,centre,use_mask", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 2])
def test_noalloc_matches_lbcg_observables(lb, name, make, centre, use_mask, precision):
    pb = make()
    sim = lb.Simulation(pb, precision)
    mask_dev = torch.from_numpy(np.ascontiguousarray(pb.mask, np.uint8)).cuda() if use_mask else None
    for call in range(2):
        # an even number of steps since binding leaves the current state in the first buffer
        sim.step(64)
        for r_in, r_out in ((-1.0, -1.0), (3.0, 8.0)):
            ref = sim.observables(centre, r_in, r_out)
            out = _noalloc(lb, sim, mask_dev, centre, r_in, r_out)
            for key in ("mass_r", "mass_b", "p_in", "p_out", "r_eff", "umax", "amount"):
                assert getattr(out, key) == pytest.approx(ref[key], rel=1e-13, abs=1e-300), (call, key)
            assert np.allclose(out.mom[:], ref["mom"], rtol=1e-13, atol=1e-13)
            assert out.dp == pytest.approx(ref["dp"], rel=1e-9, abs=1e-15)
            assert (out.n_in, out.n_out) == (ref["n_in"], ref["n_out"])
            assert out.nonfinite == 0 and out.step == -1


def test_noalloc_rejects_invalid_parameters(lb):
    pb = W.static_droplet(W.D2Q9, 16, 4)
    sim = lb.Simulation(pb, 2)
    p = lb.params_of(pb, 2)
    p.tau_r = 0.4
    L = lb.load()
    out = lb.lbcg_obs()
    c = (C.c_double * 3)(8.0, 8.0, 0.0)
    assert L.lbcg_observables_noalloc(C.byref(p), C.c_void_p(sim._a.data_ptr()), None, c, -1.0, -1.0, None,
                                      C.byref(out)) == -1
    assert L.lbcg_observables_noalloc(C.byref(sim._p), None, None, c, -1.0, -1.0, None, C.byref(out)) == -1
