"""Continuous-batching job server for many independent simulations on one GPU.

Requests (``JobSpec``) arrive over time.  The server admits them first come, first served,
while the device memory they need -- computed beforehand by ``lbm_estimate_bytes`` -- fits a
budget and a slot is free; keeps their populations resident; advances admitted jobs together in
ticks of a fixed, even number of steps (one multi-domain ``Batch`` launch sequence per tick,
rebuilt when the set of jobs changes); reads each advanced job's contact detector after the tick
with one device-to-host copy; and retires a job when it has run its step cap or, for impact
jobs, when its droplet has left the solid (contact time, Sec. III E / IV B), freeing its memory
for the next request.

Which resident jobs a tick advances is the scheduling policy.  "all": every resident job (the
GPU is shared evenly; best aggregate throughput when many jobs are resident).  "aged_srpt": the
``max_batch`` jobs with the smallest priority value, remaining work (cells x remaining steps
over the measured cell-update rate, in seconds) minus ``alpha`` times the time the job has
waited since it arrived -- short jobs finish first (low median time-to-result) and a long job's
priority rises as it waits, so it is not starved (bounded tail); the few jobs advanced together
still share one batch launch.

A job's trajectory and every observation depend only on its own inputs and on the tick length:
observations fall on job-local steps that are multiples of the tick, the batch kernels are
bitwise the single-domain kernels, and nothing crosses between jobs.  So each result is the
same whether the job runs alone or in a mix.

The scheduling logic (``Server``) is plain host code over an ``engine``; ``GpuEngine`` is the
engine that drives liblbm.so.  ``GpuEngine(batched=False)`` with ``max_active=1`` is the
one-job-at-a-time baseline.
"""
import ctypes
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from .lbm import CONTACT_FIELDS, Batch, LBMError, Simulation, estimate_bytes


@dataclass
class JobSpec:
    """One request.  make_fields() returns (rho, u, solid) host arrays in the library's layout
    (solid may be None).  The job runs until `steps` (rounded up to whole ticks) or, if
    stop_on_detach, until it has detached: after a tick with liquid-solid contact, a tick without
    from which the detector stays without contact for `detach_hold` steps (the detachment step is
    the first of those ticks).  threshold: liquid density threshold of the contact detector
    (None: no detector)."""
    name: str
    params: object
    make_fields: object
    steps: int
    stop_on_detach: bool = False
    threshold: float = None
    arrival: float = 0.0
    has_solid: bool = False
    detach_hold: int = 0


@dataclass
class JobResult:
    name: str
    status: str = "ok"
    steps: int = 0
    cells: int = 0
    touch: int = None               # first observed step with contact
    detach: int = None              # first later observed step without
    contacts: list = field(default_factory=list)   # (step, wet, floor, xmin, xmax, ymin, ymax)
    sums: tuple = None              # FP64 (sum rho, sum rho u) at the end
    populations: object = None      # final populations (host), when requested
    arrival: float = 0.0
    admitted: float = None
    finished: float = None

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival

    @property
    def contact_steps(self):
        return None if self.touch is None or self.detach is None else self.detach - self.touch


class _Slot:
    def __init__(self, spec, handle, nbytes, result):
        self.spec, self.handle, self.nbytes, self.result = spec, handle, nbytes, result
        self.step = 0
        self.done = False
        self.zero_from = None     # first tick of the current run without contact


class Server:
    """Admission, ticking and retirement over an engine (see module docstring).

    budget_bytes: device memory the resident jobs may hold; max_active: slot count;
    tick: steps per tick (even: every job stays at the even AA phase between ticks);
    policy: "all" or "aged_srpt" (with alpha, max_batch); rate: initial estimate of the
    cell updates per second, refined from every tick."""

    POLICIES = ("all", "aged_srpt")

    def __init__(self, engine, budget_bytes, tick=100, max_active=64, clock=time.perf_counter, sleep=time.sleep,
                 policy="all", alpha=4.0, max_batch=2, rate=1.6e10):
        if tick < 2 or tick % 2:
            raise ValueError("tick must be an even number of steps >= 2")
        if max_active < 1:
            raise ValueError("max_active must be >= 1")
        if policy not in self.POLICIES:
            raise ValueError(f"policy must be one of {self.POLICIES}")
        if max_batch < 1 or alpha < 0 or not rate > 0:
            raise ValueError("max_batch must be >= 1, alpha >= 0 and rate > 0")
        self.engine, self.budget, self.tick, self.max_active = engine, int(budget_bytes), int(tick), int(max_active)
        self.clock, self.sleep = clock, sleep
        self.policy, self.alpha, self.max_batch, self.rate = policy, float(alpha), int(max_batch), float(rate)
        self.stats = {}

    def select(self, active, now):
        """The resident jobs the next tick advances (see the module docstring)."""
        if self.policy == "all":
            return list(active)

        def priority(s):
            remaining = max(s.spec.steps - s.step, 0) * s.result.cells / self.rate
            return (remaining - self.alpha * (now - s.spec.arrival), s.spec.arrival)

        return sorted(active, key=priority)[:self.max_batch]

    def run(self, specs):
        """Serve `specs` (arrival times in seconds from the start of the run); returns JobResults in
        input order."""
        results = {s.name: JobResult(name=s.name, arrival=s.arrival) for s in specs}
        if len(results) != len(specs):
            raise ValueError("job names must be unique")
        pending = deque(sorted(specs, key=lambda s: s.arrival))
        for s in pending:
            need = self.engine.estimate(s)
            if need > self.budget:
                raise ValueError(f"job {s.name} needs {need} bytes, more than the budget {self.budget}")
        active = []
        used = 0
        ticks = cell_steps = 0
        busy = 0.0
        peak_bytes = peak_active = 0
        t0 = self.clock()
        while pending or active:
            now = self.clock() - t0
            # admission: first come, first served, while memory and slots allow
            while pending and pending[0].arrival <= now and len(active) < self.max_active:
                spec = pending[0]
                need = self.engine.estimate(spec)
                if used + need > self.budget:
                    break
                pending.popleft()
                res = results[spec.name]
                res.admitted = self.clock() - t0
                try:
                    handle = self.engine.admit(spec)
                except LBMError as e:
                    res.status = f"admit failed: {e}"
                    res.finished = self.clock() - t0
                    continue
                res.cells = int(spec.params.ncell)
                active.append(_Slot(spec, handle, need, res))
                used += need
            peak_bytes, peak_active = max(peak_bytes, used), max(peak_active, len(active))
            if not active:
                if pending:
                    wait = pending[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(min(wait, 0.05))
                continue
            tb = self.clock()
            run = self.select(active, tb - t0)
            handles = [s.handle for s in run]
            self.engine.advance(handles, self.tick)
            obs = self.engine.observe(handles, [s.spec.threshold for s in run])
            status = self.engine.status(handles)
            dt = self.clock() - tb
            busy += dt
            ticks += 1
            work = sum(s.result.cells for s in run) * self.tick
            if dt > 0:
                self.rate = 0.8 * self.rate + 0.2 * work / dt
            for s, o, st in zip(run, obs, status):
                s.step += self.tick
                cell_steps += s.result.cells * self.tick
                r = s.result
                r.steps = s.step
                if st is not None:
                    r.status = st
                    s.done = True
                    continue
                if o is not None:
                    r.contacts.append((s.step,) + tuple(int(v) for v in o))
                    wet = int(o[0])
                    if r.touch is None:
                        if wet > 0:
                            r.touch = s.step
                    elif r.detach is None:
                        if wet > 0:
                            s.zero_from = None
                        else:
                            if s.zero_from is None:
                                s.zero_from = s.step
                            if s.step - s.zero_from >= s.spec.detach_hold:
                                r.detach = s.zero_from
                if s.step >= s.spec.steps or (s.spec.stop_on_detach and r.detach is not None):
                    s.done = True
            still = []
            for s in active:
                if not s.done:
                    still.append(s)
                    continue
                if s.result.status == "ok":
                    s.result.sums, s.result.populations = self.engine.finish(s.handle)
                self.engine.release(s.handle)
                s.result.finished = self.clock() - t0
                used -= s.nbytes
            active = still
        wall = self.clock() - t0
        self.stats = {"wall_s": wall, "busy_s": busy, "ticks": ticks, "cell_steps": cell_steps,
                      "mlups_busy": cell_steps / busy / 1e6 if busy > 0 else 0.0,
                      "mlups_wall": cell_steps / wall / 1e6 if wall > 0 else 0.0,
                      "peak_bytes": peak_bytes, "peak_active": peak_active}
        return [results[s.name] for s in specs]


class GpuEngine:
    """Runs jobs through liblbm.so on the current CUDA device, all on one stream.

    batched=True advances the jobs of a tick with one multi-domain Batch (a lone job steps
    alone); the last `cache` batches are kept, keyed by their member set, so a scheduler that
    alternates between a few sets does not rebuild them every tick.  batched=False steps each
    job with its own single-domain launches.  keep_populations: copy every finished job's
    populations to the host (for equality checks)."""

    def __init__(self, batched=True, stream=None, keep_populations=False, cache=8):
        import torch
        from collections import OrderedDict
        self.torch = torch
        self.batched = batched
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.keep_populations = keep_populations
        self._batches = OrderedDict()
        self._cache = max(1, int(cache))
        self._obs = None
        self.launch_sets = 0

    def estimate(self, spec):
        return estimate_bytes(spec.params, with_solid=spec.has_solid)

    def admit(self, spec):
        torch = self.torch
        rho, u, solid = spec.make_fields()
        with torch.cuda.stream(self.stream):
            sim = Simulation(spec.params, stream=self.stream)
            try:
                dr = torch.as_tensor(np.ascontiguousarray(rho, dtype=np.float32)).pin_memory().to("cuda", non_blocking=True)
                du = torch.as_tensor(np.ascontiguousarray(u, dtype=np.float32)).pin_memory().to("cuda", non_blocking=True)
                ds = None
                if solid is not None:
                    ds = torch.as_tensor(np.ascontiguousarray(solid, dtype=np.uint8)).to("cuda", non_blocking=True)
                sim.init_fields(dr, du, ds)
                self.stream.synchronize()     # the temporaries are freed once the init has run
            except Exception:
                sim.close()
                raise
        return sim

    def release(self, sim):
        for key in [k for k, b in self._batches.items() if sim in b.sims]:
            self._batches.pop(key).close()
        sim.close()

    def advance(self, sims, n):
        if not self.batched or len(sims) == 1:
            # a lone job takes its own single-domain launches (the whole-grid kernels where its
            # geometry allows), faster than a one-member batch; results are the same
            for s in sims:
                s.step(n)
            self.launch_sets += len(sims)
            return
        key = tuple(sorted(id(s) for s in sims))
        b = self._batches.get(key)
        if b is None:
            while len(self._batches) >= self._cache:
                self._batches.popitem(last=False)[1].close()
            b = Batch(sims, stream=self.stream)
            self._batches[key] = b
            self.launch_sets += 1
        else:
            self._batches.move_to_end(key)
        b.step(n)

    def observe(self, sims, thresholds):
        torch = self.torch
        rows = [k for k, t in enumerate(thresholds) if t is not None]
        out = [None] * len(sims)
        if not rows:
            return out
        if self._obs is None or self._obs.shape[0] < len(rows):
            with torch.cuda.stream(self.stream):
                self._obs = torch.empty((max(len(rows), 64), 6), dtype=torch.int32, device="cuda")
        for j, k in enumerate(rows):
            sims[k].contact(thresholds[k], out=self._obs[j])
        with torch.cuda.stream(self.stream):
            host = self._obs[:len(rows)].to("cpu", non_blocking=False)
        vals = host.numpy()
        for j, k in enumerate(rows):
            out[k] = vals[j].copy()
        return out

    def status(self, sims):
        out = []
        for s in sims:
            try:
                s.sync()
                out.append(None)
            except LBMError as e:
                out.append(str(e))
        return out

    def finish(self, sim):
        sums = (ctypes.c_double * 4)()
        sim.moments_into(None, None, sums)
        pops = sim.populations(device=False) if self.keep_populations else None
        return tuple(float(v) for v in sums), pops

    def close(self):
        while self._batches:
            self._batches.popitem()[1].close()


def percentile(values, q):
    """Nearest-rank percentile (q in [0, 100]) of a non-empty list."""
    v = sorted(values)
    if not v:
        return None
    k = max(0, min(len(v) - 1, int(np.ceil(q / 100.0 * len(v))) - 1))
    return v[k]


def summary(results, stats):
    """p50 / p99 time-to-result and aggregate MLUPS of a finished run."""
    lat = [r.latency for r in results if r.status == "ok" and r.latency is not None]
    return {"jobs": len(results), "ok": len(lat), "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
            "mean_s": float(np.mean(lat)) if lat else None, **stats}


__all__ = ["CONTACT_FIELDS", "GpuEngine", "JobResult", "JobSpec", "Server", "percentile", "summary"]
