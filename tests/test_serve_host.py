"""Host logic of the job server (paper_2306_16274_gb300/serve.py) over a fake engine and a
virtual clock: admission by memory budget and slots, first-come-first-served order, retirement
at the step cap or at detachment, slot reuse, and results that do not depend on the mix."""
import numpy as np
import pytest

from paper_2306_16274_gb300.serve import JobSpec, Server, percentile, summary


class FakeParams:
    def __init__(self, ncell):
        self.ncell = ncell


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeEngine:
    """A job's wet-cell count at job-local step s is schedule[s // tick - 1]; a tick costs
    1 ms per active job plus 1 ms (so batching more jobs per tick is cheaper per job)."""

    def __init__(self, clock, tick):
        self.clock, self.tick = clock, tick
        self.resident = {}
        self.max_resident = 0
        self.admissions = []

    def estimate(self, spec):
        return spec.params.ncell * 100

    def admit(self, spec):
        h = {"spec": spec, "step": 0}
        self.resident[id(h)] = h
        self.max_resident = max(self.max_resident, len(self.resident))
        self.admissions.append(spec.name)
        return h

    def release(self, h):
        del self.resident[id(h)]

    def advance(self, hs, n):
        for h in hs:
            h["step"] += n
        self.clock.t += 0.001 * (1 + len(hs))

    def observe(self, hs, thresholds):
        out = []
        for h, t in zip(hs, thresholds):
            if t is None:
                out.append(None)
                continue
            sched = h["spec"].make_fields
            k = h["step"] // self.tick - 1
            wet = sched[k] if k < len(sched) else 0
            out.append(np.array([wet, 0, 0, 0, 0, 0], dtype=np.int32))
        return out

    def status(self, hs):
        return [None for _ in hs]

    def finish(self, h):
        return (float(h["step"]), 0.0, 0.0, float(len(h["spec"].name))), None


def job(name, ncell, steps, schedule=(), arrival=0.0, detach=True, hold=0):
    return JobSpec(name=name, params=FakeParams(ncell), make_fields=list(schedule), steps=steps,
                   stop_on_detach=detach, threshold=0.5 if schedule else None, arrival=arrival, detach_hold=hold)


def serve(specs, budget, tick=10, max_active=64):
    clock = Clock()
    eng = FakeEngine(clock, tick)
    srv = Server(eng, budget, tick=tick, max_active=max_active, clock=clock, sleep=clock.sleep)
    return srv.run(specs), srv, eng


def test_budget_and_slots_bound_the_resident_set():
    specs = [job(f"j{k}", 1000, 50, arrival=0.0) for k in range(6)]
    res, srv, eng = serve(specs, budget=250_000)            # 2.5 jobs fit: at most 2 resident
    assert eng.max_resident == 2 and srv.stats["peak_bytes"] <= 250_000
    assert all(r.status == "ok" and r.steps == 50 for r in res)
    res, srv, eng = serve(specs, budget=10 ** 9, max_active=3)
    assert eng.max_resident == 3 and srv.stats["peak_active"] == 3


def test_first_come_first_served_and_slot_reuse():
    specs = [job(f"j{k}", 1000 * (k + 1), 40, arrival=0.01 * k) for k in range(5)]
    res, srv, eng = serve(specs, budget=600_000)
    assert eng.admissions == [f"j{k}" for k in range(5)]
    admitted = [r.admitted for r in res]
    assert admitted == sorted(admitted)
    assert all(r.finished >= r.admitted >= r.arrival for r in res)


def test_retire_at_detachment_or_cap():
    specs = [job("bounce", 100, 1000, schedule=[0, 0, 7, 12, 3, 0, 0, 4]),
             job("stick", 100, 60, schedule=[0, 5, 5, 5, 5, 5, 5, 5, 5]),
             job("cap_only", 100, 35)]
    res, _, _ = serve(specs, budget=10 ** 9)
    r = {x.name: x for x in res}
    assert (r["bounce"].touch, r["bounce"].detach, r["bounce"].steps) == (30, 60, 60)
    assert r["bounce"].contact_steps == 30
    assert (r["stick"].touch, r["stick"].detach, r["stick"].steps) == (20, None, 60)
    assert r["cap_only"].steps == 40                         # rounded up to whole ticks
    assert r["cap_only"].contacts == [] and r["bounce"].contacts[2][:2] == (30, 7)


def test_detachment_needs_a_sustained_lift_off():
    # a short lift-off (one tick) is ignored with a 20-step hold; the final one counts from its start,
    # and the job stops once the hold has passed
    specs = [job("cushion", 100, 1000, schedule=[0, 3, 0, 4, 0, 0, 0, 0, 2], hold=20)]
    r = serve(specs, budget=10 ** 9)[0][0]
    assert (r.touch, r.detach, r.steps) == (20, 50, 70)
    r = serve([job("cushion0", 100, 1000, schedule=[0, 3, 0, 4, 0, 0, 0, 0, 2], hold=0)], budget=10 ** 9)[0][0]
    assert (r.touch, r.detach, r.steps) == (20, 30, 30)


def test_results_do_not_depend_on_the_mix():
    specs = [job("a", 100, 200, schedule=[0, 1, 2, 0]), job("b", 5000, 80, arrival=0.002),
             job("c", 300, 120, schedule=[0, 0, 0, 9, 9, 0], arrival=0.004)]
    together, _, _ = serve(specs, budget=10 ** 9)
    for s, t in zip(specs, together):
        alone, _, _ = serve([s], budget=10 ** 9)
        a = alone[0]
        assert (a.steps, a.touch, a.detach, a.sums, a.contacts) == (t.steps, t.touch, t.detach, t.sums, t.contacts)


def test_latency_waits_for_arrivals_and_rejects_bad_setups():
    res, srv, _ = serve([job("late", 100, 20, arrival=1.5)], budget=10 ** 9)
    assert res[0].admitted >= 1.5 and res[0].latency < 0.1
    with pytest.raises(ValueError):
        serve([job("big", 10 ** 6, 20)], budget=1000)
    with pytest.raises(ValueError):
        Server(None, 1, tick=3)
    with pytest.raises(ValueError):
        serve([job("x", 1, 2), job("x", 1, 2)], budget=10 ** 9)


def test_percentiles_and_summary():
    assert percentile([5, 1, 3, 2, 4], 50) == 3
    assert percentile(list(range(1, 101)), 99) == 99
    assert percentile([7.0], 99) == 7.0
    res, srv, _ = serve([job(f"j{k}", 100, 20, arrival=0.001 * k) for k in range(4)], budget=10 ** 9)
    s = summary(res, srv.stats)
    assert s["ok"] == 4 and s["p50_s"] <= s["p99_s"] and s["cell_steps"] == 4 * 100 * 20


class WorkEngine(FakeEngine):
    """A tick costs 1 us per cell advanced plus 0.1 ms, and the widest tick is recorded."""

    def __init__(self, clock, tick):
        super().__init__(clock, tick)
        self.widest = 0

    def advance(self, hs, n):
        for h in hs:
            h["step"] += n
        self.widest = max(self.widest, len(hs))
        self.clock.t += 1e-6 * sum(h["spec"].params.ncell for h in hs) + 1e-4


def serve_policy(specs, policy, alpha=1.0, max_batch=2, tick=10):
    clock = Clock()
    eng = WorkEngine(clock, tick)
    srv = Server(eng, 10 ** 12, tick=tick, clock=clock, sleep=clock.sleep, policy=policy, alpha=alpha,
                 max_batch=max_batch, rate=1e6)
    return {r.name: r for r in srv.run(specs)}, srv, eng


def test_aged_srpt_finishes_a_short_job_first():
    # a long job is running when a short one arrives: shared evenly ("all") the short job waits on the
    # long one's work; "aged_srpt" with one job per tick runs it at once and resumes the long one
    specs = [job("long", 10_000, 1000, detach=False), job("short", 1_000, 100, arrival=0.05, detach=False)]
    even, _, _ = serve_policy(specs, "all")
    srpt, _, eng = serve_policy(specs, "aged_srpt", alpha=0.0, max_batch=1)
    assert eng.widest == 1
    assert srpt["short"].finished < srpt["long"].finished
    assert srpt["short"].latency < even["short"].latency
    assert srpt["short"].latency < 0.11          # its own 10 ticks of 1.1 ms plus at most one tick


def test_aging_bounds_the_wait_of_a_long_job():
    # a long job and a stream of short ones arriving as fast as they are served: pure shortest-first
    # (alpha = 0) serves every short job first; with aging the long job's priority rises as it waits
    specs = [job("long", 5_000, 400, detach=False)]
    specs += [job(f"s{k}", 1_000, 30, arrival=0.002 + 0.0033 * k, detach=False) for k in range(120)]
    pure, _, _ = serve_policy(specs, "aged_srpt", alpha=0.0, max_batch=1)
    aged, _, _ = serve_policy(specs, "aged_srpt", alpha=2.0, max_batch=1)
    assert aged["long"].latency < 0.7 * pure["long"].latency


def test_policy_bounds_the_batch_and_keeps_results():
    specs = [job("a", 100, 200, schedule=[0, 1, 2, 0]), job("b", 5000, 80, arrival=0.002),
             job("c", 300, 120, schedule=[0, 0, 0, 9, 9, 0], arrival=0.004), job("d", 2000, 60)]
    ref, _, _ = serve_policy(specs, "all")
    for k in (1, 2, 3):
        got, srv, eng = serve_policy(specs, "aged_srpt", max_batch=k)
        assert eng.widest <= k
        for name, r in ref.items():
            g = got[name]
            assert (g.steps, g.touch, g.detach, g.sums, g.contacts) == (r.steps, r.touch, r.detach, r.sums, r.contacts)
    with pytest.raises(ValueError):
        Server(None, 1, policy="lifo")
    with pytest.raises(ValueError):
        Server(None, 1, policy="aged_srpt", max_batch=0)
