"""Shared helpers for the GPU parity tests: build both sides from one parameter dict,
run them on the same seeded inputs and compare element by element."""
import numpy as np

import workloads as W
from oracle import lbm as olbm

CS = W.constants()["cs"]
PW = W.constants()["piecewise"]


def cs_eos(T_key="T0.7"):
    t = CS[T_key]
    return dict(eos="cs", eos_p=(CS["a"], CS["b"], CS["R"], t["T"]), G=-1.0), t["rho_l"], t["rho_v"]


def pw_eos():
    return dict(eos="piecewise", eos_p=(PW["rho1"], PW["rho2"], PW["theta_v"], PW["theta_m"], PW["theta_l"]),
                G=-1.0), PW["rho_l"], PW["rho_v"]


def oracle_params(d):
    """oracle.lbm.Params from a plain dict (bc given as 0/1 per axis)."""
    rates = dict(olbm._mom.DEFAULT_RATES)
    rates.update(d.get("rates", {}))
    return olbm.Params(lattice=d["lattice"], shape=tuple(d["shape"]), bc=tuple(d.get("bc", (0, 0, 0))),
                       eos=d.get("eos", "none"), eos_p=tuple(d.get("eos_p", ())), G=d.get("G", -1.0),
                       G_ads=d.get("G_ads", 0.0), kappa=d.get("kappa", 0.0), sigma=d.get("sigma", 0.0),
                       rates=rates, variable_nu=d.get("variable_nu", False), nu_l=d.get("nu_l", 0.0),
                       nu_v=d.get("nu_v", 0.0), rho_l=d.get("rho_l", 1.0), rho_v=d.get("rho_v", 0.0),
                       g=tuple(d.get("g", (0.0, 0.0, 0.0))))


def gpu_params(d):
    from paper_2306_16274_gb300 import Params
    return Params(lattice=d["lattice"], shape=tuple(d["shape"]), bc=tuple(d.get("bc", (0, 0, 0))),
                  eos=d.get("eos", "none"), eos_p=tuple(d.get("eos_p", ())), G=d.get("G", -1.0),
                  G_ads=d.get("G_ads", 0.0), kappa=d.get("kappa", 0.0), sigma=d.get("sigma", 0.0),
                  rates=dict(d.get("rates", {})), variable_nu=d.get("variable_nu", False),
                  nu_l=d.get("nu_l", 0.0), nu_v=d.get("nu_v", 0.0), rho_l=d.get("rho_l", 1.0),
                  rho_v=d.get("rho_v", 0.0), g=tuple(d.get("g", (0.0, 0.0, 0.0))),
                  psi_ext_rho=d.get("psi_ext_rho", -1.0), zchunk=d.get("zchunk", 0),
                  store=d.get("store", "fp32"), onepass=d.get("onepass", False),
                  store_layout=d.get("store_layout", "auto"))


def run_gpu(d, rho, u, solid=None, steps=0, device=True):
    import torch

    from paper_2306_16274_gb300 import Simulation
    sim = Simulation(gpu_params(d))
    if device:
        args = [torch.tensor(rho, dtype=torch.float32, device="cuda"),
                torch.tensor(u, dtype=torch.float32, device="cuda"),
                None if solid is None else torch.tensor(solid, dtype=torch.uint8, device="cuda")]
    else:
        args = [rho.astype(np.float32), u.astype(np.float32), None if solid is None else solid.astype(np.uint8)]
    sim.init_fields(*args)
    if steps:
        sim.step(steps)
    return sim


def run_oracle(d, rho, u, solid=None, steps=0):
    s = olbm.State.from_fields(oracle_params(d), rho, u, None if solid is None else solid.astype(bool))
    s.u0max = float(np.abs(u).max())
    fluid = np.ones(np.shape(rho), bool) if solid is None else ~np.asarray(solid, bool)
    s.mom0 = float((np.asarray(rho) * np.sqrt((np.asarray(u) ** 2).sum(axis=0)) * fluid).sum())
    return s.run(steps)


def linf_rel(a, b):
    """max |a - b| / max |b| over the whole field (field-normwise relative L-infinity)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# every comparison made in this process: (test id, err_rho, err_u, plain L-inf of u, err of sum rho u);
# tests/conftest.py prints them at the end of the run
RECORDS = []


def _current_test():
    import os
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]


def compare_moments(sim, ref):
    """(err_rho, err_u, gpu sums, oracle sums).  err_rho = max |rho_gpu - rho_oracle| / max rho_oracle;
    err_u = max |u_gpu - u_oracle| / U with U the velocity scale of the run, the larger of the
    initial and the final max |u| of the oracle (a decaying flow keeps its initial scale).
    The plain field-relative L-infinity error of u (over the final max |u| alone) and the error of
    the FP64 momentum totals (over sum rho |u|) are recorded beside them (RECORDS)."""
    r_g, u_g, sums = sim.moments(device=True)
    r_g, u_g = r_g.cpu().numpy(), u_g.cpu().numpy()
    r_o, u_o = ref.moments()
    U = max(float(np.abs(u_o).max()), getattr(ref, "u0max", 0.0), 1e-300)
    err_u = float(np.abs(u_g.astype(np.float64) - u_o).max() / U)
    so = ref.sums()
    err_rho = linf_rel(r_g, r_o)
    RECORDS.append((_current_test(), err_rho, err_u, linf_rel(u_g, u_o), _momentum_error(sums, so, r_o, u_o, ref)))
    return err_rho, err_u, sums, so


def _momentum_error(sums_gpu, sums_oracle, r_o, u_o, ref):
    scale = max(float((r_o * np.sqrt((u_o ** 2).sum(axis=0))).sum()), getattr(ref, "mom0", 0.0), 1e-300)
    return float(np.abs(np.asarray(sums_gpu[1:]) - np.asarray(sums_oracle[1:])).max() / scale)


def momentum_error(sums_gpu, sums_oracle, ref):
    """max_a |sum rho u_a (GPU) - sum rho u_a (oracle)| over the run's momentum scale, sum rho |u| of
    the oracle at the start or at the end, whichever is larger (as for u: a decaying flow keeps the
    scale it was set up with)."""
    r_o, u_o = ref.moments()
    return _momentum_error(sums_gpu, sums_oracle, r_o, u_o, ref)
