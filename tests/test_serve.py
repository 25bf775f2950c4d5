"""Continuous-batching scheduler (host logic) with a host-only engine: admission under
the HBM budget and slot limits, first-come first-served order, completion of every
request, and the time-to-result / throughput summary."""
import numpy as np
import pytest

from paper_1711_02003_gb300 import serve
from paper_1711_02003_gb300 import workloads as W


class FakeEngine(serve.Engine):
    """Instances advance `rate` steps per advance() call; bytes = 100 per site."""

    def __init__(self, slots=3, diverging=()):
        self.slots = slots
        self.live = {}
        self.order = []
        self.n = 0
        self.evicted = []
        self.diverging = set(diverging)  # request ids whose instance goes non-finite once it runs
        self.bad = set()
        self.steps_of = {}

    def state_bytes(self, req):
        return 100 * req.problem.nsites

    def free_slots(self, lattice):
        return self.slots - sum(1 for (lat, _) in self.live.values() if lat == lattice)

    def admit(self, req):
        self.n += 1
        h = self.n
        self.live[h] = (req.problem.lattice, [req.steps])
        self.steps_of[h] = req.steps
        if req.rid in self.diverging:
            self.bad.add(h)
        self.order.append(req.rid)
        return h

    def advance(self, steps):
        for _, rem in self.live.values():
            rem[0] = max(0, rem[0] - steps)

    def finished(self):
        return [h for h, (_, rem) in self.live.items() if rem[0] == 0]

    def retire(self, h):
        self.live.pop(h)
        return {"ok": True}

    def resident(self):
        return len(self.live)

    def evict(self, h):
        self.live.pop(h)
        self.evicted.append(h)

    def diverged(self, h):
        return h in self.bad and self.live[h][1][0] < self.steps_of[h]


def reqs(n=20, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for k in range(n):
        t += rng.exponential(0.05)
        lat = int(rng.integers(0, 2))
        pb = W.Problem(lattice=lat, nx=int(rng.integers(8, 40)), ny=int(rng.integers(8, 40)), nz=1 if lat == 0 else 8,
                       mask=np.zeros(1, np.uint8))
        out.append(serve.Request(k, t, pb, int(rng.integers(50, 600))))
    return out


def test_all_complete_fifo_and_budget():
    rs = reqs()
    budget = 3 * max(100 * r.problem.nsites for r in rs)
    eng = FakeEngine(slots=2)
    srv = serve.Server(eng, hbm_budget=budget, chunk=100)
    res = srv.run(rs, realtime=False)
    assert sorted(r.rid for r in res) == list(range(len(rs)))
    assert srv.peak_used <= budget
    # first come, first served: admission order is arrival order
    assert eng.order == [r.rid for r in sorted(rs, key=lambda r: r.arrival)]
    for r in res:
        assert r.admitted >= r.arrival and r.finished >= r.admitted
    s = serve.summary(res)
    assert s["requests"] == len(rs) and s["p99_s"] >= s["p50_s"] > 0
    assert s["site_updates"] == sum(r.problem.fluid_sites() * r.steps for r in rs)


def test_request_larger_than_budget_rejected():
    rs = reqs(3)
    with pytest.raises(ValueError):
        serve.Server(FakeEngine(), hbm_budget=10.0).run(rs, realtime=False)


def test_make_requests_mix():
    rs = serve.make_requests(16, rate=20.0, seed=0, steps_scale=0.01)
    lats = {r.problem.lattice for r in rs}
    assert lats == {W.D2Q9, W.D3Q19}
    assert all(r.steps >= 1 for r in rs)
    assert np.all(np.diff([r.arrival for r in rs]) > 0)


# Failure paths, injected on the host: a client withdraws requests (before and after
# admission) and an instance diverges; each is removed with its status, its memory is
# returned to the budget, and every other request completes as before.
def test_cancelled_requests_leave_queue_and_device():
    rs = reqs(12)
    budget = 3 * max(100 * r.problem.nsites for r in rs)
    base = serve.Server(FakeEngine(slots=2), hbm_budget=budget, chunk=100).run(reqs(12), realtime=False)
    rs[2].cancel_at = 0.0                       # withdrawn while still queued
    rs[0].cancel_at = rs[0].arrival + 0.0005     # withdrawn after admission, before finishing
    eng = FakeEngine(slots=2)
    srv = serve.Server(eng, hbm_budget=budget, chunk=100)
    res = {r.rid: r for r in srv.run(rs, realtime=False)}
    assert res[2].status == "cancelled" and res[2].admitted < 0
    assert res[0].status == "cancelled" and eng.evicted
    assert srv.used == 0
    assert all(res[r.rid].status == "done" for r in base if r.rid not in (0, 2))
    s = serve.summary(list(res.values()))
    assert s["cancelled"] == 2 and s["requests"] == len(rs) - 2


def test_diverged_instance_evicted_without_disturbing_others():
    rs = reqs(10)
    budget = 3 * max(100 * r.problem.nsites for r in rs)
    eng = FakeEngine(slots=2, diverging={4})
    srv = serve.Server(eng, hbm_budget=budget, chunk=50, health_every=1)
    res = {r.rid: r for r in srv.run(rs, realtime=False)}
    assert res[4].status == "diverged"
    assert all(res[k].status == "done" for k in res if k != 4)
    assert len(res) == len(rs) and srv.used == 0
    assert serve.summary(list(res.values()))["diverged"] == 1
