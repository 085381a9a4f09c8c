"""Write workloads/constants.json from the oracle alone (test infrastructure).

Stores the Carnahan-Starling critical point and the Maxwell coexistence densities
at T = 0.7 T_c and T = 0.5 T_c for a = 0.5, b = 4, R = 1 (the static-droplet and
at-scale workloads), and the piecewise-EOS spinodal densities of Eq. e20 for
rho_v = 0.001, rho_l = 1 with the slopes of Eq. e21.  Run from the repository root:

    python -m workloads.make_constants
"""
import json
import os
import warnings

from oracle import eos


def main():
    warnings.simplefilter("ignore")
    a, b, R = 0.5, 4.0, 1.0
    rho_c, T_c = eos.cs_critical_point(a, b, R)
    out = {"cs": {"a": a, "b": b, "R": R, "rho_c": rho_c, "T_c": T_c}}
    for frac in (0.7, 0.5):
        T = frac * T_c
        rv, rl = eos.cs_maxwell(a, b, R, T)
        out["cs"][f"T{frac}"] = {"T": T, "rho_v": rv, "rho_l": rl}
    tv, tm, tl = eos.piecewise_slopes()
    r1, r2 = eos.piecewise_spinodals(0.001, 1.0, tv, tm, tl)
    out["piecewise"] = {"rho_v": 0.001, "rho_l": 1.0, "rho1": r1, "rho2": r2,
                        "theta_v": tv, "theta_m": tm, "theta_l": tl}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "constants.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
