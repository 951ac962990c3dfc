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


class ClassedExecutor(FakeExecutor):
    """Slots 0, 1 are small (fit size <= 1), slot 2 is large; a request
    marked 'overflow_small' overflows a small slot (finish returns False)."""
    sizes = (1, 1, 2)

    def fits(self, slot, req):
        return req["size"] <= self.sizes[slot]

    def slot_class(self, slot):
        return self.sizes[slot] - 1

    def finish(self, slot, req):
        super().finish(slot, req)
        req.setdefault("ran_on", []).append(slot)
        return not (req.get("overflow_small") and self.sizes[slot] == 1)


def test_admission_by_slot_class_and_bypass():
    clock = Clock(1e-4)
    ex = ClassedExecutor(clock)
    sch = Scheduler(3, ex)
    # a long large request holds the large slot; a second large one must wait
    # for it, and the small ones behind it start on the small slots meanwhile
    reqs = [{"id": 0, "arrival": 0.0, "work": 0.05, "size": 2},
            {"id": 1, "arrival": 0.001, "work": 0.01, "size": 2},
            {"id": 2, "arrival": 0.002, "work": 0.01, "size": 1},
            {"id": 3, "arrival": 0.003, "work": 0.01, "size": 1}]
    replay(sch, reqs, clock=clock)
    assert len(sch.completed) == 4
    by = {r["id"]: r for r in reqs}
    assert by[0]["slot"] == 2 and by[1]["slot"] == 2            # large only on the large slot
    assert {by[2]["slot"], by[3]["slot"]} == {0, 1}               # small prefer small slots
    assert by[2]["t_start"] < by[1]["t_start"] and by[3]["t_start"] < by[1]["t_start"]
    assert by[1]["t_start"] >= by[0]["t_start"] + 0.05 - 1e-9


def test_overflow_is_run_again_in_a_larger_class():
    clock = Clock(1e-4)
    ex = ClassedExecutor(clock)
    sch = Scheduler(3, ex)
    reqs = [{"id": i, "arrival": 0.001 * i, "work": 0.002, "size": 1,
             "overflow_small": i % 3 == 0} for i in range(12)]
    replay(sch, reqs, clock=clock)
    assert len(sch.completed) == 12 and sch.idle()
    assert sch.retries == 4
    for r in reqs:
        if r["overflow_small"]:
            assert r["retries"] == 1 and r["ran_on"][0] in (0, 1) and r["ran_on"][1] == 2
        else:
            assert "retries" not in r


def test_plan_slots_fills_the_budget_by_share():
    from paper_2503_01199_gb300.serving import plan_slots
    cost = [600, 1900, 3300]
    for budget in (5800, 9000, 14000, 40000):
        counts = plan_slots(budget, cost, [1 / 3, 1 / 3, 1 / 3])
        used = sum(c * b for c, b in zip(counts, cost))
        assert used <= budget and min(counts) >= 1
        assert all(used + b > budget for b in cost)               # nothing more fits
        assert counts[0] >= counts[2]                             # small slots at least as many
    assert plan_slots(5800, cost, [0.5, 0.5, 0.0])[2] == 0
