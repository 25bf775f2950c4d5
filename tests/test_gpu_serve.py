"""Serving on the GPU: requests of both lattices arriving over time run in the batches
(continuous batching) and each result equals the same request run alone, within the
FP32 tolerance (1e-5 relative; 1 % on the Laplace pressure)."""
import numpy as np
import pytest

from paper_1711_02003_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02003_gb300 import build
    build.build()
    from paper_1711_02003_gb300 import lbcg
    lbcg.load()
    return lbcg


def small_requests(serve, n=10):
    out = []
    t = 0.0
    for k in range(n):
        spec = W.random_request(777 + k)
        spec.update(nx=min(spec["nx"], 160), ny=min(spec["ny"], 40), nz=min(spec["nz"], 16))
        pb = W.serving_problem(spec)
        t += 0.001
        out.append(serve.Request(k, t, pb, 150 + 37 * k, (pb.nx / 2, pb.ny / 2, pb.nz / 2)))
    return out


def test_serving_results_equal_alone(lb):
    from paper_1711_02003_gb300 import serve
    rs = small_requests(serve)
    eng = serve.LbcgEngine(precision=lb.LBCG_FP32_DEV, max_slots=3)
    srv = serve.Server(eng, hbm_budget=2e9, chunk=32)
    res = srv.run(rs, realtime=True)
    assert len(res) == len(rs)
    assert srv.peak_resident >= 2          # requests overlapped on the device
    for r, q in zip(res, rs):
        sim = lb.Simulation(q.problem, lb.LBCG_FP32_DEV)
        sim.step(q.steps)
        ref = sim.observables(q.centre, allow_diverged=True)
        for key in ("mass_r", "mass_b", "p_in", "p_out", "r_eff"):
            assert r.observables[key] == pytest.approx(ref[key], rel=1e-5), (q.rid, key)
        assert r.observables["umax"] == pytest.approx(ref["umax"], rel=1e-3, abs=1e-9), q.rid
    s = serve.summary(res)
    assert s["p99_s"] >= s["p50_s"] > 0 and s["aggregate_mlups"] > 0


def test_admission_bound_by_hbm_budget(lb):
    """Six D3Q19 requests of one size under a budget that holds two of them, with eight free
    slots: the memory budget, not the slots, decides admission on the device.  Exactly two
    are resident at the peak, the resident bytes never exceed the budget, every request
    completes, and results still equal the solo runs."""
    from paper_1711_02003_gb300 import serve
    rs = []
    for k in range(6):
        spec = W.random_request(900 + k)
        spec.update(lattice=W.D3Q19, nx=96, ny=32, nz=16, geom="step" if k % 2 else "junction")
        pb = W.serving_problem(spec)
        rs.append(serve.Request(k, 0.001 * (k + 1), pb, 120 + 20 * k, (pb.nx / 2, pb.ny / 2, pb.nz / 2)))
    eng = serve.LbcgEngine(precision=lb.LBCG_FP32_DEV, max_slots=8)
    size = max(eng.state_bytes(r) for r in rs)
    assert min(eng.state_bytes(r) for r in rs) == size
    budget = 2.5 * size
    srv = serve.Server(eng, hbm_budget=budget, chunk=32)
    res = srv.run(rs, realtime=True)
    assert len(res) == len(rs)
    assert srv.peak_used <= budget
    assert srv.peak_resident == 2
    for r, q in zip(res, rs):
        sim = lb.Simulation(q.problem, lb.LBCG_FP32_DEV)
        sim.step(q.steps)
        ref = sim.observables(q.centre, allow_diverged=True)
        assert r.observables["mass_r"] == pytest.approx(ref["mass_r"], rel=1e-5), q.rid
        assert r.observables["r_eff"] == pytest.approx(ref["r_eff"], rel=1e-5), q.rid
