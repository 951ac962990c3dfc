"""Host logic of the render server (no GPU): FIFO admission onto a fixed
number of slots, completion, and the latency accounting."""
import numpy as np

from paper_2503_01199_gb300.serving import Scheduler, latency_stats, replay


class FakeExecutor:
    """A request occupies its slot for req['work'] seconds of the fake clock."""

    def __init__(self, clock):
        self.clock = clock
        self.busy_until = {}
        self.started = []

    def start(self, slot, req):
        assert slot not in self.busy_until
        self.busy_until[slot] = self.clock.t + req["work"]
        self.started.append((req["id"], slot, self.clock.t))

    def done(self, slot):
        return self.clock.t >= self.busy_until[slot]

    def finish(self, slot, req):
        del self.busy_until[slot]


class Clock:
    def __init__(self, dt):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def test_fifo_admission_never_exceeds_slots():
    clock = Clock(1e-4)
    ex = FakeExecutor(clock)
    sch = Scheduler(3, ex)
    rng = np.random.default_rng(0)
    reqs = [{"id": i, "arrival": float(a), "work": float(w)}
            for i, (a, w) in enumerate(zip(np.cumsum(rng.exponential(0.002, 200)),
                                           rng.uniform(0.001, 0.01, 200)))]
    wall = replay(sch, reqs, clock=clock)
    assert len(sch.completed) == 200 and sch.idle()
    assert sch.max_inflight == 3
    # started in arrival order, each no earlier than its arrival
    ids = [i for i, _, _ in ex.started]
    assert ids == sorted(ids)
    for r in reqs:
        assert r["t_start"] >= r["arrival"] - 1e-12 and r["t_done"] >= r["t_start"] + r["work"] - 1e-9
    # never two requests on one slot at once
    by_slot = {}
    for r in reqs:
        by_slot.setdefault(r["slot"], []).append((r["t_start"], r["t_done"]))
    for iv in by_slot.values():
        iv.sort()
        assert all(a[1] <= b[0] + 1e-12 for a, b in zip(iv, iv[1:]))
    st = latency_stats(reqs, wall)
    lat = np.array([r["t_done"] - r["arrival"] for r in reqs]) * 1e3
    assert st["requests"] == 200 and abs(st["p50_ms"] - np.percentile(lat, 50)) < 1e-3
    assert st["p99_ms"] >= st["p50_ms"]


def test_requests_arriving_while_busy_wait_for_a_free_slot():
    clock = Clock(1e-4)
    ex = FakeExecutor(clock)
    sch = Scheduler(1, ex)
    reqs = [{"id": i, "arrival": 0.0, "work": 0.01} for i in range(4)]
    replay(sch, reqs, clock=clock)
    starts = [r["t_start"] for r in reqs]
    assert all(b - a >= 0.01 - 1e-9 for a, b in zip(starts, starts[1:]))
    assert sch.max_inflight == 1
