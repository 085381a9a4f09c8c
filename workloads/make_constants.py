"""Write workloads/constants.json from the oracle alone (test infrastructure).

Stores the Carnahan-Starling critical point and the Maxwell coexistence densities
at T = 0.7 T_c and T = 0.5 T_c for a = 0.5, b = 4, R = 1 (the static-droplet and
at-scale workloads), the surface tension at 0.7 T_c for kappa = 0 and 0.3 (Laplace's law,
used to set impact velocities and capillary times), and the piecewise-EOS spinodal densities of Eq. e20 for
rho_v = 0.001, rho_l = 1 with the slopes of Eq. e21.  Run from the repository root:

    python -m workloads.make_constants
"""
import json
import os
import warnings

import numpy as np

import workloads
from oracle import eos, lbm


def planar_equilibrium(cs, steps=10000):
    """Relax a planar liquid slab (160 x 1 x 1, D3Q19, C-S at T = 0.5 T_c, G = -1, sigma = 0.1,
    kappa = 0.5, s2b = 1.0) with the oracle and return its coexistence densities and the interface
    width W = (rho_l - rho_v) / max |d rho / dx| of Eq. e23: the model's own equilibrium, used to
    start droplets near equilibrium in the large-density-ratio workload."""
    t = cs["T0.5"]
    rates = dict(lbm._mom.DEFAULT_RATES)
    rates["s2b"] = 1.0
    p = lbm.Params(lattice=19, shape=(160, 1, 1), eos="cs", eos_p=(cs["a"], cs["b"], cs["R"], t["T"]), G=-1.0,
                   sigma=0.1, kappa=0.5, rates=rates)
    rho, u = workloads.slab((160, 1, 1), 80, t["rho_l"], t["rho_v"], W=5.0)
    s = lbm.State.from_fields(p, rho, u).run(steps)
    r = s.moments()[0][0, 0]
    return {"rho_l": float(r.max()), "rho_v": float(r.min()),
            "W": float((r.max() - r.min()) / np.abs(np.diff(r)).max()), "steps": steps,
            "setup": "D3Q19 slab 160x1x1, sigma=0.1, kappa=0.5, s2b=1.0"}


def column_surface_tension(cs, kappa, steps=1000):
    """Surface tension of the C-S fluid at T = 0.7 T_c (D3Q19, G = -1, sigma = 0.1, default
    rates) from Laplace's law on a liquid column (Sec. III C): gamma = (p_in - p_out) R, the mean
    over R = 8 and R = 12 in a 48 x 48 x 1 periodic box after `steps` steps, pressures from the
    EOS at the column centre and the far corner."""
    t = cs["T0.7"]
    vals = []
    for R in (8, 12):
        p = lbm.Params(lattice=19, shape=(48, 48, 1), eos="cs", eos_p=(cs["a"], cs["b"], cs["R"], t["T"]), G=-1.0,
                       sigma=0.1, kappa=kappa)
        s = lbm.State.from_fields(p, *workloads.cylinder_droplet((48, 48, 1), R, t["rho_l"], t["rho_v"])).run(steps)
        r = s.moments()[0][0]
        pin = eos.cs_pressure(r[24, 24], cs["a"], cs["b"], cs["R"], t["T"])
        pout = eos.cs_pressure(r[0, 0], cs["a"], cs["b"], cs["R"], t["T"])
        vals.append((pin - pout) * R)
    return float(np.mean(vals))


def main():
    warnings.simplefilter("ignore")
    a, b, R = 0.5, 4.0, 1.0
    rho_c, T_c = eos.cs_critical_point(a, b, R)
    out = {"cs": {"a": a, "b": b, "R": R, "rho_c": rho_c, "T_c": T_c}}
    for frac in (0.7, 0.6, 0.55, 0.5):
        T = frac * T_c
        rv, rl = eos.cs_maxwell(a, b, R, T)
        out["cs"][f"T{frac}"] = {"T": T, "rho_v": rv, "rho_l": rl}
    tv, tm, tl = eos.piecewise_slopes()
    r1, r2 = eos.piecewise_spinodals(0.001, 1.0, tv, tm, tl)
    out["piecewise"] = {"rho_v": 0.001, "rho_l": 1.0, "rho1": r1, "rho2": r2,
                        "theta_v": tv, "theta_m": tm, "theta_l": tl}
    out["cs"]["planar_T0.5"] = planar_equilibrium(out["cs"])
    out["cs"]["gamma_T0.7"] = {f"kappa{k}": column_surface_tension(out["cs"], k) for k in (0.0, 0.3)}
    out["cs"]["gamma_T0.7"]["setup"] = "Laplace column 48x48x1, R = 8 and 12, 1000 steps, D3Q19, sigma = 0.1"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "constants.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
