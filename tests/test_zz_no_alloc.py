"""lbcg_observables_noalloc: the allocation-free observables entry point.

Some callers cannot allocate device memory (plug-ins whose host application owns every
allocation through its own pool, loops that forbid allocation after start-up, code running
with the device memory budget fully committed).  This entry point needs no context and keeps
its reduction scratch in a file-scope device array.  These checks call it through the C ABI
on the buffer that holds a context's current state and compare it with lbcg_observables on
the same state, in every storage precision and twice in a row (the shared scratch carries
nothing from one call into the next), on a lattice large enough that the reduction grid is
capped and its blocks stride over the sites, and on a stream that is being captured: the
call is synchronous, so it must refuse there and leave the capture intact."""
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
    # 327,680 sites: more than 1024 blocks of 256 sites, so the grid is capped and strides
    ("droplet D2Q9 640x512", lambda: W.static_droplet(W.D2Q9, 640, 100, ny=512), (320, 256, 0), False),
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


def _call(lb, sim, mask_dev, centre, r_in=-1.0, r_out=-1.0, stream=None):
    L = lb.load()
    out = lb.lbcg_obs()
    c = (C.c_double * 3)(*[float(v) for v in centre])
    st = (stream or sim.stream).cuda_stream
    status = L.lbcg_observables_noalloc(C.byref(sim._p), C.c_void_p(sim.current_state_ptr),
                                        None if mask_dev is None else C.c_void_p(mask_dev.data_ptr()), c,
                                        float(r_in), float(r_out), C.c_void_p(st), C.byref(out))
    return status, out


def _noalloc(lb, sim, mask_dev, centre, r_in=-1.0, r_out=-1.0):
    status, out = _call(lb, sim, mask_dev, centre, r_in, r_out)
    assert status == 0, lb.load().lbcg_last_error().decode()
    return out


@pytest.mark.parametrize("name,make,centre,use_mask", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_noalloc_matches_lbcg_observables(lb, name, make, centre, use_mask, precision):
    pb = make()
    sim = lb.Simulation(pb, precision)
    mask_dev = torch.from_numpy(np.ascontiguousarray(pb.mask, np.uint8)).cuda() if use_mask else None
    for call, steps in enumerate((33, 64)):   # odd, then even: the current state is in either buffer
        sim.step(steps)
        for r_in, r_out in ((-1.0, -1.0), (3.0, 8.0)):
            ref = sim.observables(centre, r_in, r_out)
            out = _noalloc(lb, sim, mask_dev, centre, r_in, r_out)
            for key in ("mass_r", "mass_b", "p_in", "p_out", "r_eff", "umax", "amount"):
                assert getattr(out, key) == pytest.approx(ref[key], rel=1e-13, abs=1e-300), (call, key)
            assert np.allclose(out.mom[:], ref["mom"], rtol=1e-13, atol=1e-13)
            assert out.dp == pytest.approx(ref["dp"], rel=1e-9, abs=1e-15)
            assert (out.n_in, out.n_out) == (ref["n_in"], ref["n_out"])
            assert out.nonfinite == 0 and out.step == -1


def test_noalloc_refuses_a_capturing_stream(lb):
    pb = W.static_droplet(W.D2Q9, 32, 8)
    sim = lb.Simulation(pb, lb.LBCG_FP32_DEV)
    sim.step(3)
    before = _noalloc(lb, sim, None, (16, 16, 0))
    x = torch.zeros(4, device="cuda")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        x.add_(1.0)
        status, _ = _call(lb, sim, None, (16, 16, 0), stream=side)
    assert status == lb.LBCG_ERR_STATE, status
    assert "captured" in lb.load().lbcg_last_error().decode()
    graph.replay()
    torch.cuda.synchronize()
    assert x.tolist() == [1.0] * 4          # the capture ended cleanly and replays
    after = _noalloc(lb, sim, None, (16, 16, 0))
    assert after.mass_r == before.mass_r and after.dp == before.dp


def test_noalloc_rejects_invalid_parameters(lb):
    pb = W.static_droplet(W.D2Q9, 16, 4)
    sim = lb.Simulation(pb, 2)
    p = lb.params_of(pb, 2)
    p.tau_r = 0.4
    L = lb.load()
    out = lb.lbcg_obs()
    c = (C.c_double * 3)(8.0, 8.0, 0.0)
    assert L.lbcg_observables_noalloc(C.byref(p), C.c_void_p(sim.current_state_ptr), None, c, -1.0, -1.0, None,
                                      C.byref(out)) == -1
    assert L.lbcg_observables_noalloc(C.byref(sim._p), None, None, c, -1.0, -1.0, None, C.byref(out)) == -1
