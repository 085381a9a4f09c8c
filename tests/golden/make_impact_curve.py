"""Write tests/golden/impact_curve.json: the spreading diameter D_f(t) of a droplet hitting a flat
wall, computed by the FP64 oracle alone (test infrastructure; imports only oracle/ and workloads/).

Down-scaled counterpart of the paper's droplet impact on a wall (Sec. III E / IV A): D3Q19,
100 x 100 x 50 cells, walls in z (half-way bounce-back), periodic in x and y, neutral wall
(G_ads = 0, 90 degrees), the piecewise EOS of Eqs. e19-e21 (rho_v = 0.001, rho_l = 1), G = -1,
sigma = 0.1, kappa = 0, droplet R0 = 12.5 two cells above the wall (tanh width 4) falling at
U = 0.08, nu = 0.05 (s2 = 1 / (3 nu + 1/2)), s4 = 1 (the paper's s4 = 1.2 makes D3Q19 unstable at
low viscosity), other rates as in the paper.  D_f is the mean of the x and y extents of liquid
(rho > (rho_l + rho_v) / 2) in the first fluid layer above the wall, sampled every 25 steps up to
t* = U t / R0 = 3.

    python -m tests.golden.make_impact_curve
"""
import json
import os
import sys
import time

import numpy as np

import workloads as W
from oracle import lbm, observe

SHAPE = (100, 100, 50)
R0, U, NU, EVERY, STEPS = 12.5, 0.08, 0.05, 25, 475


def params():
    pw = W.constants()["piecewise"]
    rates = dict(lbm._mom.DEFAULT_RATES)
    rates["s2"] = 1.0 / (3.0 * NU + 0.5)
    rates["s4"] = 1.0
    return lbm.Params(lattice=19, shape=SHAPE, bc=(0, 0, 1), eos="piecewise",
                      eos_p=(pw["rho1"], pw["rho2"], pw["theta_v"], pw["theta_m"], pw["theta_l"]), G=-1.0,
                      sigma=0.1, kappa=0.0, rates=rates)


def fields():
    pw = W.constants()["piecewise"]
    return W.impact(SHAPE, R0, pw["rho_l"], pw["rho_v"], U=U, gap=2.0, W=4.0)


def main():
    pw = W.constants()["piecewise"]
    thr = 0.5 * (pw["rho_l"] + pw["rho_v"])
    s = lbm.State.from_fields(params(), *fields())
    t0 = time.time()
    steps, df, wet = [], [], []
    for k in range(STEPS // EVERY):
        s.run(EVERY)
        rho = s.moments()[0]
        c = observe.contact(rho, None, (0, 0, 1), 19, thr)
        steps.append(s.t)
        df.append(observe.spreading_diameter(c))
        wet.append(c[0])
        print(s.t, df[-1], round(time.time() - t0), flush=True, file=sys.stderr)
    out = {"setup": __doc__.split("\n\n")[1].replace("\n", " "), "R0": R0, "U": U, "nu": NU, "shape": SHAPE,
           "every": EVERY, "steps": steps, "D_f": df, "wet": wet,
           "mass": float(s.sums()[0]), "oracle_seconds": round(time.time() - t0, 1)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "impact_curve.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
