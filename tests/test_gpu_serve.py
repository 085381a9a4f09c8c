"""Contact detector and memory estimate against the oracle's definitions, and the job server's
promise: every job's result is the same alone and in a mix of concurrently served jobs."""
import numpy as np
import pytest

import workloads as W
from oracle import observe
from tests import parity_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def impact_case(Q, shape, ratio, steps, bc=(0, 0, 1), G_ads=0.23):
    kw, rl, rv = U.cs_eos("T0.7")
    R0 = min(shape[0], shape[1]) / 6.0
    rho, u, solid = W.cylinder_impact(shape, R0, ratio * R0, rl, rv, U=0.08, gap=2.0)
    d = dict(lattice=Q, shape=shape, bc=bc, sigma=0.1, kappa=0.3, G_ads=G_ads, **kw)
    return d, rho, u, solid, 0.5 * (rl + rv)


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("ratio", [0.5, 1.5])
def test_contact_matches_oracle_definition_on_gpu_density(Q, ratio):
    d, rho, u, solid, thr = impact_case(Q, (48, 40, 52), ratio, 0)
    sim = U.run_gpu(d, rho, u, solid)
    seen_contact = False
    for _ in range(6):
        sim.step(40)
        r, _, _ = sim.moments(device=False)
        got = sim.contact(thr)
        want = observe.contact(r, solid, (0, 0, 1), Q, thr)
        assert [got[k] for k in ("wet", "floor", "xmin", "xmax", "ymin", "ymax")] == want
        seen_contact |= want[0] > 0
    assert seen_contact


def test_contact_floor_footprint_and_device_output():
    import torch
    kw, rl, rv = U.cs_eos("T0.7")
    shape = (40, 36, 30)
    rho, u = W.impact(shape, 8.0, rl, rv, U=0.05, gap=1.0)
    d = dict(lattice=19, shape=shape, bc=(0, 0, 1), sigma=0.1, kappa=0.3, **kw)
    sim = U.run_gpu(d, rho, u)
    thr = 0.5 * (rl + rv)
    sim.step(120)
    r, _, _ = sim.moments(device=False)
    want = observe.contact(r, None, (0, 0, 1), 19, thr)
    assert want[1] > 0                        # the droplet has spread on the floor
    host = sim.contact(thr)
    assert list(host.values()) == want
    buf = torch.full((3, 6), -7, dtype=torch.int32, device="cuda")
    sim.contact(thr, out=buf[1])
    torch.cuda.synchronize()
    assert buf[1].cpu().tolist() == want and buf[0].cpu().tolist() == [-7] * 6
    # no walls, no solids: nothing can touch
    d2 = dict(lattice=19, shape=(16, 16, 16), sigma=0.1, **kw)
    sim2 = U.run_gpu(d2, *W.droplet((16, 16, 16), 4.0, rl, rv))
    assert sim2.contact(thr) == {"wet": 0, "floor": 0, "xmin": 2 ** 31 - 1, "xmax": -2 ** 31,
                                 "ymin": 2 ** 31 - 1, "ymax": -2 ** 31}


@pytest.mark.parametrize("Q,with_solid", [(19, False), (27, True)])
def test_estimate_equals_device_bytes(Q, with_solid):
    from paper_2306_16274_gb300 import estimate_bytes
    d, rho, u, solid, _ = impact_case(Q, (33, 29, 41), 1.0, 0)
    sim = U.run_gpu(d, rho, u, solid if with_solid else None)
    assert sim.device_bytes == estimate_bytes(U.gpu_params(d), with_solid=with_solid)
    n = 33 * 29 * 41
    sim.moments(device=False)                 # host copy: a 4-float-per-cell staging buffer appears
    assert sim.device_bytes == estimate_bytes(U.gpu_params(d), with_solid=with_solid) + 16 * n


def _specs(arrivals):
    from paper_2306_16274_gb300.serve import JobSpec
    specs = []
    cases = [("imp19a", 19, (48, 40, 52), 0.5), ("imp27", 27, (40, 44, 46), 1.2), ("imp19b", 19, (36, 36, 40), 2.0)]
    for (name, Q, shape, ratio), t in zip(cases, arrivals):
        d, rho, u, solid, thr = impact_case(Q, shape, ratio, 0)
        specs.append(JobSpec(name=name, params=U.gpu_params(d), make_fields=lambda r=rho, v=u, s=solid: (r, v, s),
                             steps=400, stop_on_detach=True, threshold=thr, arrival=t, has_solid=True))
    kw, rl, rv = U.cs_eos("T0.7")
    for (name, Q, L, R, kappa), t in zip([("drop19", 19, 30, 7.0, 0.0), ("drop27", 27, 26, 6.0, 0.3)], arrivals[3:]):
        d = dict(lattice=Q, shape=(L, L, L), sigma=0.1, kappa=kappa, **kw)
        rho, u = W.droplet((L, L, L), R, rl, rv)
        specs.append(JobSpec(name=name, params=U.gpu_params(d), make_fields=lambda r=rho, v=u: (r, v, None),
                             steps=300, arrival=t))
    return specs


def test_each_result_is_the_same_alone_and_in_the_mix():
    from paper_2306_16274_gb300.serve import GpuEngine, Server
    mix = Server(GpuEngine(batched=True, keep_populations=True), budget_bytes=2 ** 33, tick=20)
    together = mix.run(_specs([0.0, 0.0, 0.004, 0.0, 0.002]))
    assert mix.stats["peak_active"] >= 3     # the jobs overlapped on the device
    for spec, t in zip(_specs([0.0] * 5), together):
        solo = Server(GpuEngine(batched=False, keep_populations=True), budget_bytes=2 ** 33, tick=20)
        a = solo.run([spec])[0]
        assert a.status == t.status == "ok"
        assert (a.steps, a.touch, a.detach) == (t.steps, t.touch, t.detach)
        assert a.contacts == t.contacts
        assert a.sums == t.sums
        assert np.array_equal(a.populations, t.populations)


def test_each_result_is_the_same_under_the_aged_srpt_scheduler():
    # the scheduler advances two of the resident jobs per tick, chosen anew each tick (batches of
    # alternating pairs come from the engine's cache): every result is still the job's alone
    from paper_2306_16274_gb300.serve import GpuEngine, Server
    eng = GpuEngine(batched=True, keep_populations=True, cache=2)
    mix = Server(eng, budget_bytes=2 ** 33, tick=20, policy="aged_srpt", alpha=1.0, max_batch=2, rate=2e9)
    together = mix.run(_specs([0.0, 0.0, 0.004, 0.0, 0.002]))
    assert mix.stats["peak_active"] >= 3 and eng.launch_sets >= 2
    for spec, t in zip(_specs([0.0] * 5), together):
        solo = Server(GpuEngine(batched=False, keep_populations=True), budget_bytes=2 ** 33, tick=20)
        a = solo.run([spec])[0]
        assert a.status == t.status == "ok"
        assert (a.steps, a.touch, a.detach, a.contacts, a.sums) == (t.steps, t.touch, t.detach, t.contacts, t.sums)
        assert np.array_equal(a.populations, t.populations)


def test_budget_limits_residency_on_the_gpu():
    from paper_2306_16274_gb300 import estimate_bytes
    from paper_2306_16274_gb300.serve import GpuEngine, Server
    specs = _specs([0.0] * 5)
    need = sorted(estimate_bytes(s.params, s.has_solid) for s in specs)
    budget = need[-1] + need[-2]              # any two jobs fit, three of the largest do not
    srv = Server(GpuEngine(batched=True), budget_bytes=budget, tick=20)
    res = srv.run(specs)
    assert all(r.status == "ok" for r in res)
    assert srv.stats["peak_bytes"] <= budget and srv.stats["peak_active"] <= 4
