"""Batched execution (lbcg_batch_*): every instance's populations equal its solo run
within rounding (the batched kernel runs the same per-site code; the compiler may
contract multiply-adds differently in it), whatever the mix, the step counts, or when
the instance was admitted."""
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


TOL = {0: 1e-13, 2: 2e-6}   # max |difference| of populations: FP64, FP32-dev


def problems_2d():
    return [W.cross_junction(nx=130, channel_w=16, side_x=40, side_len=12, fill_x=30),
            W.static_droplet(W.D2Q9, 61, 12, ny=37, tau_r=1.5, tau_b=0.8),
            W.channel(W.D2Q9, 96, 20, U=0.01, outlet=W.PRESSURE_OUTLET, two_phase=True, A=0.01),
            W.cross_junction(nx=200, channel_w=24, side_x=60, side_len=16, u_disp=0.004, fill_x=50)]


def problems_3d():
    return [W.step_emulsifier(nx=70, ny=20, nz=12, terrace_len=24, terrace_h=4, u_in=0.01, fill_x=12),
            W.static_droplet(W.D3Q19, 24, 6.5, ny=20, nz=18, centre=(11.5, 9.5, 8.5)),
            W.step_emulsifier(nx=50, ny=30, nz=10, terrace_len=20, terrace_h=4, u_in=0.005, fill_x=10)]


@pytest.mark.parametrize("lattice", [0, 1])
@pytest.mark.parametrize("precision", [0, 2])
def test_batch_equals_alone(lb, lattice, precision):
    probs = problems_2d() if lattice == 0 else problems_3d()
    steps = [37, 64, 101, 5][:len(probs)]
    alone = []
    for pb, n in zip(probs, steps):
        s = lb.Simulation(pb, precision)
        s.step(n)
        alone.append(s.populations())
    batch = lb.Batch(lattice, precision, max_instances=8)
    sims = [lb.Simulation(pb, precision, stream=batch.stream) for pb in probs]
    slots = [batch.add(s, n) for s, n in zip(sims, steps)]
    batch.step(1000)
    done = sorted(batch.poll())
    assert done == sorted(slots)
    for s, ref, n in zip(sims, alone, steps):
        assert s.step_count == n
        d = np.abs(s.populations() - ref).max()
        assert d <= TOL[precision], d


def test_continuous_admission_equals_alone(lb):
    """Instances admitted while others run (and retired as they finish) match solo runs."""
    probs = problems_2d()
    plan = [(0, 0, 90), (1, 0, 40), (2, 20, 70), (3, 50, 33)]  # (problem, admitted at, steps)
    alone = {}
    for k, t0, n in plan:
        s = lb.Simulation(probs[k], lb.LBCG_FP32_DEV)
        s.step(n)
        alone[k] = s.populations()
    batch = lb.Batch(0, lb.LBCG_FP32_DEV, max_instances=3)
    sims, pending, t = {}, list(plan), 0
    finished = {}
    while pending or batch.active:
        for item in [p for p in pending if p[1] <= t]:
            if batch.active < 3:
                k, _, n = item
                sims[k] = lb.Simulation(probs[k], lb.LBCG_FP32_DEV, stream=batch.stream)
                sims[k].slot = batch.add(sims[k], n)
                pending.remove(item)
        batch.step(10)
        t += 10
        for slot in batch.poll():
            k = next(k for k, s in sims.items() if getattr(s, "slot", None) == slot and k not in finished)
            finished[k] = sims[k].populations()
            batch.remove(slot)
    for k in alone:
        d = np.abs(finished[k] - alone[k]).max()
        assert d <= TOL[2], (k, d)


def test_batch_rejects_mismatch(lb):
    batch = lb.Batch(0, lb.LBCG_FP32_DEV, max_instances=1)
    s3 = lb.Simulation(problems_3d()[0], lb.LBCG_FP32_DEV, stream=batch.stream)
    with pytest.raises(lb.LbcgError):
        batch.add(s3, 10)
    s2 = lb.Simulation(problems_2d()[1], lb.LBCG_FP32_DEV, stream=batch.stream)
    batch.add(s2, 10)
    with pytest.raises(lb.LbcgError):
        batch.add(lb.Simulation(problems_2d()[1], lb.LBCG_FP32_DEV, stream=batch.stream), 10)
