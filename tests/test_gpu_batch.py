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


def state(pops, pb):
    """Populations with port ghost sites zeroed: a ghost is refilled from its inward neighbour
    before every step, and between steps holds the refill of an earlier state (solo D3Q19 steps
    refill the next state as they write it, batched steps the current one before stepping)."""
    out = pops.copy()
    if pb.mask is not None:
        out[:, :, np.asarray(pb.mask).ravel() >= W.PORT0] = 0.0
    return out


def problems_2d():
    return [W.cross_junction(nx=130, channel_w=16, side_x=40, side_len=12, fill_x=30),
            W.static_droplet(W.D2Q9, 61, 12, ny=37, tau_r=1.5, tau_b=0.8),
            W.channel(W.D2Q9, 96, 20, U=0.01, outlet=W.PRESSURE_OUTLET, two_phase=True, A=0.01),
            W.cross_junction(nx=200, channel_w=24, side_x=60, side_len=16, u_disp=0.004, fill_x=50)]


def problems_3d():
    return [W.step_emulsifier(nx=70, ny=20, nz=12, terrace_len=24, terrace_h=4, u_in=0.01, fill_x=12),
            W.static_droplet(W.D3Q19, 24, 6.5, ny=20, nz=18, centre=(11.5, 9.5, 8.5)),
            W.step_emulsifier(nx=50, ny=30, nz=10, terrace_len=20, terrace_h=4, u_in=0.005, fill_x=10)]


SHAPES = {0: [None, dict(rows=7, strips_per_item=3, blocks_per_sm=2, graph_steps=12)],
          1: [None, dict(rows=5, block_rows=6, blocks_per_sm=1, graph_steps=16)]}


@pytest.mark.parametrize("shape", [0, 1], ids=["default-shape", "other-shape"])
@pytest.mark.parametrize("lattice", [0, 1])
@pytest.mark.parametrize("precision", [0, 2])
def test_batch_equals_alone(lb, lattice, precision, shape):
    probs = problems_2d() if lattice == 0 else problems_3d()
    steps = [37, 64, 101, 5][:len(probs)]
    alone = []
    for pb, n in zip(probs, steps):
        s = lb.Simulation(pb, precision)
        s.step(n)
        alone.append(state(s.populations(), pb))
    batch = lb.Batch(lattice, precision, max_instances=8, shape=SHAPES[lattice][shape])
    if SHAPES[lattice][shape]:
        got = batch.shape
        want = SHAPES[lattice][shape]
        assert all(got[k] == v for k, v in want.items() if k != "blocks_per_sm"), got
        assert 1 <= got["blocks_per_sm"] <= want["blocks_per_sm"] and got["sms"] > 0  # clamped to what fits
    sims = [lb.Simulation(pb, precision, stream=batch.stream) for pb in probs]
    slots = [batch.add(s, n) for s, n in zip(sims, steps)]
    batch.step(1000)
    done = sorted(batch.poll())
    assert done == sorted(slots)
    for s, ref, n, pb in zip(sims, alone, steps, probs):
        assert s.step_count == n
        d = np.abs(state(s.populations(), pb) - ref).max()
        assert d <= TOL[precision], d
    # a batched instance resumed on its own continues like an instance never batched
    ref = lb.Simulation(probs[0], precision)
    ref.step(steps[0] + 9)
    sims[0].step(9)
    assert np.abs(state(sims[0].populations(), probs[0]) - state(ref.populations(), probs[0])).max() <= TOL[precision]


def test_continuous_admission_equals_alone(lb):
    """Instances admitted while others run (and retired as they finish) match solo runs."""
    probs = problems_2d()
    plan = [(0, 0, 90), (1, 0, 40), (2, 20, 70), (3, 50, 33)]  # (problem, admitted at, steps)
    alone = {}
    for k, t0, n in plan:
        s = lb.Simulation(probs[k], lb.LBCG_FP32_DEV)
        s.step(n)
        alone[k] = state(s.populations(), probs[k])
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
            finished[k] = state(sims[k].populations(), probs[k])
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


@pytest.mark.parametrize("lattice", [0, 1])
def test_shape_change_mid_run_is_bit_identical(lb, lattice):
    """Re-cutting the instances of a running batch (lbcg_batch_set_shape) changes nothing in the
    per-site arithmetic: the result equals a run under one shape bit for bit."""
    probs = problems_2d()[:3] if lattice == 0 else problems_3d()
    other = SHAPES[lattice][1]

    def run(switch):
        batch = lb.Batch(lattice, lb.LBCG_FP32_DEV, max_instances=4)
        sims = [lb.Simulation(pb, lb.LBCG_FP32_DEV, stream=batch.stream) for pb in probs]
        for s in sims:
            batch.add(s, 90)
        batch.step(40)
        if switch:
            batch.set_shape(**other)
        batch.step(50)
        batch.poll()
        return [state(s.populations(), pb) for s, pb in zip(sims, probs)]
    for a, b in zip(run(False), run(True)):
        assert np.array_equal(a, b)


def test_batch_autotune_picks_a_valid_shape(lb):
    from paper_1711_02003_gb300 import autotune
    res = autotune.autotune_batch(problems_3d(), lb.LBCG_FP32_DEV, steps=16,
                                  cands=[dict(rows=8, block_rows=8), dict(rows=4, block_rows=6)], graph_steps=(16,))
    assert res["mlups"] > 0 and len(res["table"]) == 3
    assert res["shape"]["block_rows"] in (6, 8) and res["shape"]["graph_steps"] in (16, 32)
