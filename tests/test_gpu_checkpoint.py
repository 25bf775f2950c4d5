"""Checkpoint / resume: n steps, save, load into a fresh context, n more steps gives the
same state, bit for bit, as 2n uninterrupted steps (every storage precision)."""
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


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
@pytest.mark.parametrize("make", [lambda: W.cross_junction(nx=130, channel_w=16, side_x=40, side_len=12, fill_x=30),
                                  lambda: W.step_emulsifier(nx=50, ny=30, nz=10, terrace_len=20, terrace_h=4,
                                                            u_in=0.01, fill_x=10)], ids=["junction2d", "step3d"])
def test_resume_is_exact(lb, tmp_path, precision, make):
    pb = make()
    n = 33
    whole = lb.Simulation(pb, precision)
    whole.step(2 * n)
    first = lb.Simulation(pb, precision)
    first.step(n)
    path = str(tmp_path / "ck.npz")
    first.save(path)
    resumed = lb.Simulation.load(path, pb)
    assert resumed.total_steps == n
    resumed.step(n)
    assert resumed.total_steps == 2 * n
    assert np.array_equal(resumed.populations(), whole.populations())


def test_library_checkpoint_file(lb, tmp_path):
    pb = W.cross_junction(nx=130, channel_w=16, side_x=40, side_len=12, fill_x=30)
    a = lb.Simulation(pb, lb.LBCG_FP32_DEV)
    a.step(21)
    path = str(tmp_path / "ck.lbcg")
    a.save_file(path)
    b = lb.Simulation(pb, lb.LBCG_FP32_DEV, init=False)
    b.load_file(path)
    assert b.step_count == 21
    a.step(21)
    b.step(21)
    assert np.array_equal(a.populations(), b.populations())
    other = lb.Simulation(W.static_droplet(W.D2Q9, 32, 8), lb.LBCG_FP32_DEV)
    with pytest.raises(lb.LbcgError):
        other.load_file(path)
