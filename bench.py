"""Benchmark of the fused non-orthogonal MRT pseudopotential step on GB300.

Workload (the paper's method at scale, one domain per GPU): 256^3 periodic,
Carnahan-Starling EOS (a = 0.5, b = 4, R = 1) at T = 0.6 T_c with the Maxwell
coexistence densities, random sphere droplets (radii uniform in [10, 40],
numpy seed 2306, liquid fraction >= 0.10) in vapour, surface-tension tuning
kappa = 0.5, sigma = 0.1, the paper's default relaxation rates, FP32
populations.  The headline value is D3Q19
MLUPS; the D3Q27 lattice is measured in the same run and reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica of the domain
(independent problems: weak scaling, no collective on the data path); the
timed region is bracketed by barriers and the maximum over ranks is used.
Prints one JSON line on rank 0.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "MLUPS & % HBM peak (fused MRT-pseudopotential step); batched p50/p99 job latency"
UNIT = "MLUPS"
SHAPE = (256, 256, 256)
WORKLOAD = ("256^3 periodic, C-S EOS (a=0.5,b=4,R=1) at T=0.6Tc (at 0.5Tc the start-up pressure wave compresses "
            "the centre of the smallest droplet past the C-S range within 20 steps), Maxwell coexistence "
            "densities (ratio 132), "
            "random sphere droplets r~U[10,40] (seed 2306, liquid fraction>=0.10, tanh W=3), kappa=0.5, "
            "sigma=0.1, G=-1, the paper's default rates, FP32 populations (AA in place)")


NOMINAL_HBM_GBS = 8000.0   # HBM3e data-sheet bandwidth, for context beside the measured copy peak


def algorithmic_bytes(Q, store="fp32", onepass=False):
    """Bytes per cell update that the method must move: collide-stream reads and writes the Q
    populations and reads psi once (8Q + 4); the density/psi pass reads the Q populations and
    writes psi (4Q + 4).  Shifted FP16 store: 2-byte slots, and the density field the slots are
    relative to is read by both passes and written by the density pass (collide 4Q + 12,
    density/psi 2Q + 12).  One-pass stepping over two copies: the Q populations read and written
    once (8Q); psi never leaves the chip."""
    if onepass:
        return {"collide": 8 * Q, "psi": 0, "step": 8 * Q}
    if store == "fp16":
        return {"collide": 4 * Q + 12, "psi": 2 * Q + 12, "step": 6 * Q + 24}
    return {"collide": 8 * Q + 4, "psi": 4 * Q + 4, "step": 12 * Q + 8}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload_fields(shape, scale=1.0, temperature="T0.6", r_min=10.0):
    """Random sphere droplets in vapour between the Maxwell coexistence densities of the C-S EOS at
    the given temperature, tanh interfaces (W = 3 at 0.6 T_c, 2 at 0.7 T_c), kappa = 0.5,
    sigma = 0.1, G = -1 and the paper's default relaxation rates."""
    c = W.constants()["cs"]
    t = c[temperature]
    width = 3.0 if temperature == "T0.6" else 2.0
    rho, u, spheres = W.random_spheres(shape, t["rho_l"], t["rho_v"], r_min * scale,
                                       40.0 * scale, seed=2306, target_fraction=0.10, gap=4.0, W=width)
    params = dict(eos="cs", eos_p=(c["a"], c["b"], c["R"], t["T"]), G=-1.0, sigma=0.1, kappa=0.5)
    return rho, u, params


# ---------------------------------------------------------------- clocks sampling
class Clocks:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        if which == 0:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for (t, line) in self.lines:
            if self.t0 is not None and not (self.t0 - 0.05 <= t <= (self.t1 or t) + 0.15):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- distributed helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, local):
    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return dist
    return None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value, device="cuda"):
    """Largest value over all ranks (the slowest replica sets the job time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world_size, cells, steps, ms_max):
    """Whole-job throughput of N replicas: all ranks' cell updates over the slowest rank's time."""
    return world_size * cells * steps / (ms_max * 1e-3) / 1e6


# ---------------------------------------------------------------- our arm
def run_lattice(Q, rho, u, wparams, steps, warmup, dist, clocks=None, store="fp32", onepass=False):
    import torch

    from paper_2306_16274_gb300 import Params, Simulation
    p = Params(lattice=Q, shape=SHAPE, store=store, onepass=onepass, **wparams)
    stream = torch.cuda.Stream()
    sim = Simulation(p, stream=stream)
    with torch.cuda.stream(stream):
        sim.init_fields(torch.tensor(rho, dtype=torch.float32, device="cuda"),
                        torch.tensor(u, dtype=torch.float32, device="cuda"))
        sim.step(warmup)
        sim.sync()
        _, _, sums0 = sim.moments()
        sim.set_kernel_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(dist)
        torch.cuda.synchronize()
        if clocks:
            clocks.mark(0)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        if clocks:
            clocks.mark(1)
        barrier(dist)
        ms = e0.elapsed_time(e1)
        kms, klaunch = sim.kernel_timing()
        sim.set_kernel_timing(False)
        sim.sync()
        _, _, sums1 = sim.moments()
    n = float(np.prod(SHAPE))
    out = dict(ms=ms, kernel_ms=kms, kernel_launches=klaunch, mass_drift=float(abs(sums1[0] - sums0[0]) / sums0[0]),
               device_bytes=sim.device_bytes)
    sim.close()
    del sim
    torch.cuda.synchronize()
    out["mlups_local"] = n * steps / (ms * 1e-3) / 1e6
    return out


def run_e2e(Q, rho, u, wparams, steps, dist=None, ws=1):
    """Same metric through the public API with host buffers: pinned host -> device fields,
    `steps` steps, device -> host moments and sums, timed by the host clock around the whole job
    (every rank its own replica between barriers; whole-job rate over the slowest rank)."""
    import torch

    from paper_2306_16274_gb300 import Params, Simulation
    n = int(np.prod(SHAPE))
    rho_h = torch.tensor(rho, dtype=torch.float32).pin_memory()
    u_h = torch.tensor(u, dtype=torch.float32).pin_memory()
    rho_o = torch.empty(n, dtype=torch.float32).pin_memory()
    u_o = torch.empty(3 * n, dtype=torch.float32).pin_memory()
    stream = torch.cuda.Stream()
    sim = Simulation(Params(lattice=Q, shape=SHAPE, **wparams), stream=stream)
    import ctypes
    sums = (ctypes.c_double * 4)()
    torch.cuda.synchronize()
    barrier(dist)
    t0 = time.perf_counter()
    sim.init_fields(rho_h, u_h)
    sim.step(steps)
    sim.moments_into(rho_o, u_o, sums)
    t1 = time.perf_counter()
    barrier(dist)
    sim.close()
    seconds = max_over_ranks(dist, t1 - t0)
    h2d = 4 * n * 4
    d2h = 4 * n * 4 + 4 * 8
    return dict(value=ws * n * steps / seconds / 1e6, unit=UNIT, h2d_bytes_per_step=h2d / steps,
                d2h_bytes_per_step=d2h / steps, seconds=seconds)


# ---------------------------------------------------------------- batched jobs
BATCH_WORKLOAD = ("64 independent jobs, cubic edge L ~ U{48..160} (numpy seed 2306), lattice D3Q19/D3Q27 and job "
                  "type by fair coin: static droplet (periodic, R = L/4) or droplet impact on a flat wall (walls in z, "
                  "R = L/5, 3 cells above the wall, U = 0.02), C-S at 0.7 T_c, sigma = 0.1, kappa = 0.3, FP32")


def batch_jobs(n_jobs=64, seed=2306):
    c = W.constants()["cs"]
    t = c["T0.7"]
    eos = dict(eos="cs", eos_p=(c["a"], c["b"], c["R"], t["T"]), G=-1.0, sigma=0.1, kappa=0.3)
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(n_jobs):
        L = int(rng.integers(48, 161))
        Q = 19 if rng.random() < 0.5 else 27
        impact = rng.random() < 0.5
        if impact:
            rho, u = W.impact((L, L, L), L / 5.0, t["rho_l"], t["rho_v"], U=0.02, gap=3.0)
            params = dict(lattice=Q, shape=(L, L, L), bc=("periodic", "periodic", "wall"), **eos)
        else:
            rho, u = W.droplet((L, L, L), L / 4.0, t["rho_l"], t["rho_v"])
            params = dict(lattice=Q, shape=(L, L, L), **eos)
        jobs.append((params, rho, u))
    return jobs


def run_batched(steps, n_jobs=64):
    """The same jobs advanced one at a time (each job's `steps` steps through the plain single-domain
    kernels, jobs back to back) and together (one tuned batch, one graph launch)."""
    import torch

    from paper_2306_16274_gb300 import Batch, Params, Simulation
    jobs = batch_jobs(n_jobs)
    stream = torch.cuda.Stream()
    sims, inputs = [], []
    with torch.cuda.stream(stream):
        for params, rho, u in jobs:
            sims.append(Simulation(Params(**params), stream=stream))
            inputs.append((torch.tensor(rho, dtype=torch.float32, device="cuda"),
                           torch.tensor(u, dtype=torch.float32, device="cuda")))

        def reset():
            for s, (r, uu) in zip(sims, inputs):
                s.init_fields(r, uu)

        cells = float(sum(np.prod(p["shape"]) for p, _, _ in jobs))
        byts = float(sum(np.prod(p["shape"]) * (12 * p["lattice"] + 8) for p, _, _ in jobs))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # one job at a time
        reset()
        for s in sims:
            s.step(2)
        torch.cuda.synchronize()
        e0.record(stream)
        for s in sims:
            s.step(steps)
        e1.record(stream)
        e1.synchronize()
        loop_ms = e0.elapsed_time(e1)
        for s in sims:
            s.sync()
        # together
        reset()
        batch = Batch(sims, stream=stream)
        choice = batch.tune(trial_steps=2)
        batch.step(2)
        torch.cuda.synchronize()
        e0.record(stream)
        batch.step(steps)
        e1.record(stream)
        e1.synchronize()
        batch_ms = e0.elapsed_time(e1)
        batch.sync()
        info = batch.info()
        shapes = [g["shape"] for g in batch.groups()]
        batch.close()
        for s in sims:
            s.close()
    torch.cuda.synchronize()
    return {"workload": BATCH_WORKLOAD, "jobs": n_jobs, "cells": int(cells), "steps": steps,
            "gpu_bytes": int(sum(np.prod(p["shape"]) * (4 * p["lattice"] + 4) for p, _, _ in jobs)),
            "one_at_a_time": {"mlups": cells * steps / (loop_ms * 1e-3) / 1e6, "ms": loop_ms},
            "batched": {"mlups": cells * steps / (batch_ms * 1e-3) / 1e6, "ms": batch_ms,
                        "hbm_frac": byts * steps / (batch_ms * 1e-3) / 1e9 / measured_peaks()[0],
                        "groups": info["groups"], "tiles": info["tiles"], "graph_mode": info["graph_mode"],
                        "zchunk": choice, "tile_shapes": shapes, "launches_per_step": 2 * info["groups"]},
            "speedup": loop_ms / batch_ms}


# ---------------------------------------------------------------- serving (continuous batching)
SERVE_WORKLOAD = ("request stream of {n} jobs (numpy seed 2306; scheduler under Poisson arrivals: aged shortest-remaining-"
                  "work first, alpha = {alpha} s/s, {k} jobs per tick; all resident jobs per tick when all arrive at "
                  "once): by fair coin droplet impact on a wall with a cylinder "
                  "(Sec. IV B; edge L ~ U{{64..160}}, R0 = L/6, R/R0 ~ U[0.2, 2], cylinder on the bottom wall along y, "
                  "walls in z, G_ads = 0.23, We = 10 from the oracle's Laplace surface tension, nu = 0.05, tanh width 3, "
                  "run until "
                  "the droplet has left the solid for 0.3 capillary times, at most 4 capillary times) or a static droplet of a kappa sweep "
                  "(periodic L^3, R ~ U[L/8, L/4], kappa in 0..0.6, 2000 steps); lattice D3Q19/D3Q27 by fair coin; "
                  "C-S at 0.7 T_c, sigma = 0.1; ticks of 100 steps; budget 150 GB")


_FIELDS = {}


def serving_specs(n_jobs, rate, seed=2306):
    """JobSpecs of the serving workload, arrivals Poisson with `rate` per second (0: all at once).
    Fields are generated once per job (the client's side of a request) and handed over as float32."""
    from paper_2306_16274_gb300 import Params
    from paper_2306_16274_gb300.serve import JobSpec
    c = W.constants()["cs"]
    t = c["T0.7"]
    rl, rv = t["rho_l"], t["rho_v"]
    gamma = c["gamma_T0.7"]["kappa0.3"]
    eos = dict(eos="cs", eos_p=(c["a"], c["b"], c["R"], t["T"]), G=-1.0, sigma=0.1)
    specs = []
    for k, j in enumerate(W.serving_jobs(n_jobs, rate, seed=seed)):
        if j["kind"] == "impact":
            R0 = j["R0"]
            U = (10.0 * gamma / (rl * R0)) ** 0.5            # We = rho_l R0 U^2 / gamma = 10
            tau = (rl * R0 ** 3 / gamma) ** 0.5              # capillary time of Sec. III E
            p = Params(lattice=j["lattice"], shape=j["shape"], bc=("periodic", "periodic", "wall"), kappa=0.3,
                       G_ads=0.23, rates={"s2": 1.0 / (3 * 0.05 + 0.5)}, **eos)
            if j["name"] not in _FIELDS:
                rho, u, solid = W.cylinder_impact(j["shape"], R0, j["Rc"], rl, rv, U, gap=3.0, W=3.0)
                _FIELDS[j["name"]] = (rho.astype(np.float32), u.astype(np.float32), solid)
            f = _FIELDS[j["name"]]
            specs.append(JobSpec(name=j["name"], params=p, make_fields=lambda f=f: f, steps=int(4 * tau),
                                 stop_on_detach=True, threshold=0.5 * (rl + rv), arrival=j["arrival"],
                                 has_solid=True, detach_hold=int(0.3 * tau)))
        else:
            p = Params(lattice=j["lattice"], shape=j["shape"], kappa=0.15 * (k % 5), **eos)
            if j["name"] not in _FIELDS:
                rho, u = W.droplet(j["shape"], j["R"], rl, rv)
                _FIELDS[j["name"]] = (rho.astype(np.float32), u.astype(np.float32), None)
            f = _FIELDS[j["name"]]
            specs.append(JobSpec(name=j["name"], params=p, make_fields=lambda f=f: f, steps=2000,
                                 arrival=j["arrival"]))
    return specs


SERVE_ALPHA, SERVE_BATCH = 4.0, 2

BUDGET_WORKLOAD = ("admission under the memory budget: {n} droplet-on-cylinder impact requests at once (numpy seed "
                   "2306), edge L ~ U{{96..256}}, height raised to fit cylinder and droplet, R0 = L/6, R/R0 ~ "
                   "U[0.2, 2], G_ads = 0.23, We = 10, nu = 0.05, C-S 0.7 T_c, lattice by fair coin, {steps} steps "
                   "each, fields generated per request at admission; budget {budget:.0f} GB")


def budget_specs(n_jobs, steps, seed=2306):
    """Impact requests over the full domain range, all at t = 0, each capped at `steps` steps;
    make_fields builds a request's fields when the server admits it (host memory stays bounded)."""
    from paper_2306_16274_gb300 import Params
    from paper_2306_16274_gb300.serve import JobSpec
    c = W.constants()["cs"]
    t = c["T0.7"]
    rl, rv = t["rho_l"], t["rho_v"]
    gamma = c["gamma_T0.7"]["kappa0.3"]
    eos = dict(eos="cs", eos_p=(c["a"], c["b"], c["R"], t["T"]), G=-1.0, sigma=0.1)
    specs = []
    for j in W.serving_jobs(n_jobs, 0.0, seed=seed, edge=(96, 256), impact_fraction=1.0):
        R0 = j["R0"]
        U = (10.0 * gamma / (rl * R0)) ** 0.5
        p = Params(lattice=j["lattice"], shape=j["shape"], bc=("periodic", "periodic", "wall"), kappa=0.3,
                   G_ads=0.23, rates={"s2": 1.0 / (3 * 0.05 + 0.5)}, **eos)

        def make(j=j, R0=R0, U=U):
            rho, u, solid = W.cylinder_impact(j["shape"], R0, j["Rc"], rl, rv, U, gap=3.0, W=3.0)
            return rho.astype(np.float32), u.astype(np.float32), solid

        specs.append(JobSpec(name=j["name"], params=p, make_fields=make, steps=steps, arrival=0.0, has_solid=True))
    return specs


def run_serving_budget(n_jobs=320, steps=200, budget=150e9):
    """More impact requests over the full domain range than the budget holds, all at once, batched
    (every resident job each tick): the budget, not the slot count, bounds the resident set."""
    import torch

    from paper_2306_16274_gb300 import estimate_bytes
    from paper_2306_16274_gb300.serve import GpuEngine, Server, summary
    specs = budget_specs(n_jobs, steps)
    need = sum(estimate_bytes(s.params, s.has_solid) for s in specs)
    eng = GpuEngine(batched=True)
    srv = Server(eng, budget, tick=100, max_active=10 ** 6)
    res = srv.run(specs)
    eng.close()
    torch.cuda.synchronize()
    out = summary(res, srv.stats)
    cells = [int(np.prod(s.params.shape)) for s in specs]
    return {"workload": BUDGET_WORKLOAD.format(n=n_jobs, steps=steps, budget=budget / 1e9), "jobs": n_jobs,
            "requested_bytes": need, "budget_bytes": budget, "peak_bytes": out["peak_bytes"],
            "peak_active": out["peak_active"], "cells_min": min(cells), "cells_max": max(cells),
            "mlups_busy": out["mlups_busy"], "mlups_wall": out["mlups_wall"], "busy_s": out["busy_s"],
            "wall_s": out["wall_s"], "ok": out["ok"], "failed": [r.name + ": " + r.status for r in res if r.status != "ok"]}


def run_serving(n_jobs=64, load=0.8, tick=100, budget=150e9):
    """The request stream served one job at a time (single-domain kernels, first come first served)
    and with continuous batching: first all requests at t = 0, every resident job advanced each tick
    (throughput); then Poisson arrivals at `load` times the one-at-a-time service rate measured in
    the first run (time-to-result), batched with the aged shortest-remaining-work scheduler, and for
    context with every resident job advanced each tick."""
    import torch

    from paper_2306_16274_gb300.serve import GpuEngine, Server, summary

    def serve(specs, batched, policy="all"):
        eng = GpuEngine(batched=batched)
        srv = Server(eng, budget, tick=tick, max_active=64 if batched else 1, policy=policy, alpha=SERVE_ALPHA,
                     max_batch=SERVE_BATCH)
        res = srv.run(specs)
        eng.close()
        torch.cuda.synchronize()
        out = summary(res, srv.stats)
        out["failed"] = [r.name + ": " + r.status for r in res if r.status != "ok"]
        return out, res

    def same(ra, rb):
        return all(a.steps == b.steps and a.touch == b.touch and a.detach == b.detach and a.sums == b.sums
                   for a, b in zip(ra, rb))

    closed = serving_specs(n_jobs, 0.0)
    seq_c, seq_res = serve(closed, False)
    bat_c, bat_res = serve(closed, True)
    rate = load * n_jobs / seq_c["busy_s"]
    open_ = serving_specs(n_jobs, rate)
    seq_o, _ = serve(open_, False)
    bat_o, bat_o_res = serve(open_, True, "aged_srpt")
    all_o, _ = serve(open_, True)
    keep = ("p50_s", "p99_s", "mean_s", "wall_s", "busy_s", "mlups_busy", "mlups_wall", "peak_active", "peak_bytes",
            "ok", "failed")
    tc = [r.contact_steps for r in bat_res if r.contact_steps is not None]
    return {"workload": SERVE_WORKLOAD.format(n=n_jobs, alpha=SERVE_ALPHA, k=SERVE_BATCH), "jobs": n_jobs,
            "cell_steps": seq_c["cell_steps"],
            "results_equal_alone_and_batched": same(seq_res, bat_res) and same(seq_res, bat_o_res),
            "all_at_once": {"one_at_a_time": {k: seq_c[k] for k in keep},
                            "batched": {k: bat_c[k] for k in keep},
                            "mlups_ratio": bat_c["mlups_wall"] / seq_c["mlups_wall"]},
            "poisson": {"rate_per_s": rate, "load": load,
                        "one_at_a_time": {k: seq_o[k] for k in keep}, "batched": {k: bat_o[k] for k in keep},
                        "policy": f"aged_srpt alpha={SERVE_ALPHA} max_batch={SERVE_BATCH}",
                        "p50_ratio": seq_o["p50_s"] / bat_o["p50_s"], "p99_ratio": seq_o["p99_s"] / bat_o["p99_s"],
                        "mlups_busy_ratio": bat_o["mlups_busy"] / seq_o["mlups_busy"],
                        "batched_all_resident": {k: all_o[k] for k in keep}},
            "impacts_detached": len(tc)}


# ---------------------------------------------------------------- oracle timing on host cores
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import bench, workloads as W
from oracle import lbm
shape = {shape!r}
rho, u, wp = bench.workload_fields(shape, scale={scale!r}, r_min=5.0 / {scale!r})
rates = dict(lbm._mom.DEFAULT_RATES)
p = lbm.Params(lattice={Q}, shape=shape, eos="cs", eos_p=tuple(wp["eos_p"]), G=-1.0, sigma=0.1, kappa=0.5,
               rates=rates)
s = lbm.State.from_fields(p, rho, u)
w0 = time.perf_counter()
for _ in range(max(1, {warmup})):        # untimed warm-up steps, at most a quarter of the budget
    s.step()
    if time.perf_counter() - w0 > 0.25 * {budget!r}:
        break
steps, t0 = 0, time.perf_counter()
times = []
while True:
    a = time.perf_counter(); s.step(); times.append(time.perf_counter() - a); steps += 1
    if time.perf_counter() - t0 > {budget!r} or steps >= {max_steps}:
        break
el = time.perf_counter() - t0
n = shape[0] * shape[1] * shape[2]
print(json.dumps(dict(steps=steps, seconds=el, mlups=n * steps / el / 1e6, step_times=times)))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_timing(Q, budget, max_steps=10 ** 9, shape=(64, 64, 64), warmup=1, procs=1):
    """FP64 oracle steps of a copy of the workload: `procs` independent processes of one thread each
    (one per host core), each `warmup` untimed steps, then timed steps until `max_steps` or `budget`
    seconds (whichever comes first).  Returns the aggregate rate (sum over processes) and the
    per-process records."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    code = ORACLE_SNIPPET.format(root=ROOT, shape=shape, scale=shape[0] / SHAPE[0], Q=Q, budget=float(budget),
                                 max_steps=int(max_steps), warmup=int(warmup))
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           env=env) for _ in range(max(1, procs))]
    runs = []
    for pr in ps:
        try:
            out, err = pr.communicate(timeout=budget + 600)
        except subprocess.TimeoutExpired:
            for q in ps:
                q.kill()
            raise RuntimeError("oracle timing did not finish")
        if pr.returncode != 0:
            raise RuntimeError("oracle timing failed: " + err[-2000:])
        runs.append(json.loads(out.strip().splitlines()[-1]))
    return {"mlups": sum(r["mlups"] for r in runs), "steps": sum(r["steps"] for r in runs),
            "seconds": max(r["seconds"] for r in runs), "procs": len(runs),
            "mlups_per_process": [r["mlups"] for r in runs], "step_ms": 1e3 * sum(r["seconds"] for r in runs) /
            max(1, sum(r["steps"] for r in runs))}


REFERENCE_SECONDS = 150.0


def reference_arm(args, ws, rank):
    if rank != 0:
        return
    Q = 19
    shape = (64, 64, 64)
    # the FP64 oracle as it stands, one replica per host core, bounded to about three minutes in all
    cores = host_cores()
    r = oracle_timing(Q, budget=REFERENCE_SECONDS, max_steps=args.steps, shape=shape, warmup=args.warmup,
                      procs=cores)
    value = r["mlups"]
    sample = (f"{cores} independent one-thread replicas of the FP64 oracle (one per host core), each on a "
              f"{shape[0]}^3 copy of the workload (radii U[5,10]): {r['steps']} timed steps in all (at most "
              f"{args.steps} and {REFERENCE_SECONDS:.0f} s per replica) after {args.warmup} warm-up steps; "
              f"value = the sum of the replicas' rates")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["step_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " -- oracle sample: 64^3 copies (radii U[5,10]), one per host core",
                       "lattice": Q, "shape": list(shape)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- traffic from the committed ncu summary
def committed_traffic(Q):
    """dram bytes per launch of the collide kernel from profiles/collide_q{Q}_traffic.json, if present
    and recorded for the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"collide_q{Q}_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    try:
        import hashlib
        src = open(os.path.join(ROOT, "paper_2306_16274_gb300", "csrc", "kernels_impl.cuh"), "rb").read()
        src += open(os.path.join(ROOT, "paper_2306_16274_gb300", "csrc", "lbm_device.cuh"), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != d.get("kernel_source_sha256_16"):
            return None
        cells_full = float(np.prod(SHAPE))
        return d["dram_bytes_per_launch"] * cells_full / d["cells"]
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-q27", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=2000)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-fp16", action="store_true")
    ap.add_argument("--no-onepass", action="store_true")
    ap.add_argument("--serving-jobs", type=int, default=64)
    ap.add_argument("--serving-budget", action="store_true",
                    help="also run the admission leg over the full domain range (minutes of host-side field generation)")
    ap.add_argument("--temperature", default="0.6", choices=["0.6", "0.7"],
                    help="T / T_c of the C-S EOS; 0.7 only for profiling cases")
    ap.add_argument("--size", type=int, default=256,
                    help="cubic edge; anything but 256 is a profiling case, not the benchmark workload")
    args = ap.parse_args()
    global SHAPE
    if args.size != 256:
        SHAPE = (args.size,) * 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, ws, rank)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import torch
    import __graft_entry__
    __graft_entry__.build()
    dist = init_dist(ws, local)
    torch.cuda.set_device(local)
    rho, u, wparams = workload_fields(SHAPE, scale=SHAPE[0] / 256.0, temperature="T" + args.temperature)
    n = float(np.prod(SHAPE))
    peak, peak_kind = measured_peaks()

    clocks = Clocks(local) if rank == 0 else None
    if clocks:
        clocks.start()
    r19 = run_lattice(19, rho, u, wparams, args.steps, args.warmup, dist, clocks)
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(dist, r19["ms"])
    value = whole_job_mlups(ws, n, args.steps, ms)
    # the side legs characterise one GPU; with several ranks only the headline and e2e run
    single = ws == 1
    r27 = None if (args.no_q27 or not single) else run_lattice(27, rho, u, wparams, args.steps, args.warmup, dist)
    e2e = None if args.no_e2e else run_e2e(19, rho, u, wparams, args.steps, dist, ws)
    f16 = {} if (args.no_fp16 or not single) else {
        Q: run_lattice(Q, rho, u, wparams, args.steps, args.warmup, dist, store="fp16")
                                   for Q in ((19,) if args.no_q27 else (19, 27))}
    one = {} if (args.no_onepass or not single) else {
        Q: run_lattice(Q, rho, u, wparams, args.steps, args.warmup, dist, onepass=True)
                                   for Q in ((19,) if args.no_q27 else (19, 27))}
    batched = None if (args.no_batched or not single or SHAPE != (256, 256, 256)) else run_batched(args.batched_steps)
    serving = None if (args.no_serving or not single or SHAPE != (256, 256, 256)) else run_serving(args.serving_jobs)
    budget_leg = run_serving_budget() if (args.serving_budget and single) else None
    if rank != 0:
        return
    ab = algorithmic_bytes(19)
    coll_ms = r19["kernel_ms"]["collide"] / max(r19["kernel_launches"]["collide"], 1)
    psi_ms = r19["kernel_ms"]["psi"] / max(r19["kernel_launches"]["psi"], 1)
    achieved = ab["collide"] * n / (coll_ms * 1e-3) / 1e9
    traffic = committed_traffic(19)
    step_gbs = ab["step"] * n * args.steps / (r19["ms"] * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if (SHAPE == (256, 256, 256) and args.temperature == "0.6")
                   else f"PROFILING CASE {SHAPE} T={args.temperature}Tc",
                   "lattice": 19, "shape": list(SHAPE), "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (populations %.2f GB per domain)" % (19 * 4 * n / 1e9)},
        "hbm_frac_step": step_gbs / peak,
        "roofline": {"kernel": "collide_kernel (fused collide-stream, D3Q19)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_cell": ab["collide"], "avg_launch_ms": coll_ms,
                     "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS},
        "kernels": {"collide": {"avg_ms": coll_ms, "launches": r19["kernel_launches"]["collide"],
                                "gbs": achieved},
                    "psi": {"avg_ms": psi_ms, "launches": r19["kernel_launches"]["psi"],
                            "gbs": ab["psi"] * n / (psi_ms * 1e-3) / 1e9 if psi_ms > 0 else None}},
        "gpu_launches": int(r19["kernel_launches"]["collide"] + r19["kernel_launches"]["psi"]),
        "mass_drift_rel": r19["mass_drift"],
        "clocks": clk,
    }
    if r27:
        ab27 = algorithmic_bytes(27)
        c27 = r27["kernel_ms"]["collide"] / max(r27["kernel_launches"]["collide"], 1)
        p27 = r27["kernel_ms"]["psi"] / max(r27["kernel_launches"]["psi"], 1)
        line["d3q27"] = {"value": r27["mlups_local"], "unit": UNIT, "ms_per_step": r27["ms"] / args.steps,
                         "hbm_frac_step": ab27["step"] * n * args.steps / (r27["ms"] * 1e-3) / 1e9 / peak,
                         "collide_gbs": ab27["collide"] * n / (c27 * 1e-3) / 1e9, "collide_avg_ms": c27,
                         "psi_gbs": ab27["psi"] * n / (p27 * 1e-3) / 1e9 if p27 > 0 else None,
                         "psi_avg_ms": p27, "mass_drift_rel": r27["mass_drift"]}
    if e2e:
        line["e2e"] = e2e
    if f16:
        line["fp16_store"] = {"note": "shifted FP16 population store (FP32 arithmetic); accuracy against the FP64 "
                                      "oracle is checked per result by tests/test_gpu_fp16.py"}
        for Q, r in f16.items():
            abh = algorithmic_bytes(Q, "fp16")
            cms = r["kernel_ms"]["collide"] / max(r["kernel_launches"]["collide"], 1)
            pms = r["kernel_ms"]["psi"] / max(r["kernel_launches"]["psi"], 1)
            line["fp16_store"][f"d3q{Q}"] = {
                "value": r["mlups_local"], "unit": UNIT, "ms_per_step": r["ms"] / args.steps,
                "bytes_per_cell": abh["step"],
                "hbm_frac_step": abh["step"] * n * args.steps / (r["ms"] * 1e-3) / 1e9 / peak,
                "collide_gbs": abh["collide"] * n / (cms * 1e-3) / 1e9,
                "psi_gbs": abh["psi"] * n / (pms * 1e-3) / 1e9, "mass_drift_rel": r["mass_drift"],
                "device_bytes": r["device_bytes"]}
    if one:
        line["onepass"] = {"note": "one pass per step over two population copies (same results bit for bit, "
                                   "tests/test_gpu_onepass.py); twice the population memory"}
        for Q, r in one.items():
            ab1 = algorithmic_bytes(Q, onepass=True)
            cms = r["kernel_ms"]["collide"] / max(r["kernel_launches"]["collide"], 1)
            line["onepass"][f"d3q{Q}"] = {
                "value": r["mlups_local"], "unit": UNIT, "ms_per_step": r["ms"] / args.steps,
                "bytes_per_cell": ab1["step"],
                "hbm_frac_step": ab1["step"] * n * args.steps / (r["ms"] * 1e-3) / 1e9 / peak,
                "kernel_gbs": ab1["collide"] * n / (cms * 1e-3) / 1e9, "kernel_avg_ms": cms,
                "mass_drift_rel": r["mass_drift"], "device_bytes": r["device_bytes"]}
    if batched:
        line["batched"] = batched
    if budget_leg:
        line["serving_budget"] = budget_leg
    if serving:
        line["serving"] = serving
        po = serving.get("poisson", {})
        if "batched" in po and "one_at_a_time" in po:
            # the metric's second part: time-to-result of the request stream under Poisson arrivals
            line["job_latency"] = {
                "unit": "s", "arrivals": "Poisson at 0.8 of the one-at-a-time service rate",
                "scheduler": po.get("policy"),
                "batched": {"p50": po["batched"]["p50_s"], "p99": po["batched"]["p99_s"],
                            "mean": po["batched"]["mean_s"]},
                "one_at_a_time": {"p50": po["one_at_a_time"]["p50_s"], "p99": po["one_at_a_time"]["p99_s"],
                                  "mean": po["one_at_a_time"]["mean_s"]}}
    if ws == 1 and not args.no_cpu_baseline:
        try:
            cores = host_cores()
            cb = oracle_timing(19, args.cpu_seconds, procs=cores)
            c1 = oracle_timing(19, args.cpu_seconds)
            line["cpu_baseline"] = {"value": cb["mlups"], "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"{cores} independent one-thread replicas of the FP64 oracle (one "
                                              f"per host core), each on a 64^3 copy of the workload (radii "
                                              f"U[5,10]) for {args.cpu_seconds:.0f} s: {cb['steps']} steps in "
                                              f"all; value = the sum of the replicas' rates",
                                    "single_thread": {"value": c1["mlups"], "cores": 1, "steps": c1["steps"],
                                                      "seconds": c1["seconds"]}}
        except Exception as exc:  # the baseline is context; never lose the GPU line over it
            line["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
