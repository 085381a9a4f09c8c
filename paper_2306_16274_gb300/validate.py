"""Physics validation of the GPU path against the values the paper prints (Sec. III).

Every case runs through the public API (Simulation / Batch) on the current CUDA device and is
measured on the host from the fields the library returns; pressures come from the library's own
psi (p = rho c_s^2 + G psi^2 / 2 with c = 1, the mechanical pressure the square-root
pseudopotential is built to reproduce, Sec. II C).  The fluid is the paper's: piecewise-linear
EOS with rho_v = 0.001, rho_l = 1 (Eqs. e19-e21), G = -1, sigma = 0.1.

  X1  planar interface: coexistence densities and interface width (Sec. III A)
  X2  static droplet: liquid density as at the planar interface, density ratio (Sec. III A)
  X4  spurious velocities in the vapour vs viscosity, MRT vs SRT (Sec. III B, Table I)
  X5  Laplace's law at several kappa: gamma vs (1 - kappa) (Sec. III C, Fig. 2a/b), D3Q19 and D3Q27
  X6  capillary-wave periods vs the dispersion relation (Sec. III C, Fig. 2c)
  X7  spatial convergence of the steady densities (Sec. III D; meshes 100-300 instead of 100-400)
  X8  contact time of a droplet bouncing off a super-hydrophobic wall (Sec. III E, Eq. e24)
  C3  droplet impact on a wall at full size (400 x 400 x 200, R0 = 50): spreading diameter with
      FP32 populations and with the shifted-FP16 store (the 4x down-scaled copy is compared with
      the oracle in tests/test_gpu_impact_curve.py)

    python -m paper_2306_16274_gb300.validate [--quick] [--cases X1,X5,...]

prints one JSON line per case on stderr as it finishes and one JSON object with everything on
stdout.
"""
import argparse
import json
import math
import sys
import time

import numpy as np

from .lbm import Batch, Params, Simulation

# fluid of Sec. III A (Eqs. e19-e21): rho_v = 0.001, rho_l = 1, slopes theta_v = 1/6, theta_m = -1/120,
# theta_l = 1/3; the spinodal densities are the roots of Eq. e20 (printed after Eq. e21: 0.001325, 0.9758)
RHO_V, RHO_L = 0.001, 1.0
PIECEWISE = (0.0013246030524049143, 0.9758004064414756, 1.0 / 6.0, -1.0 / 120.0, 1.0 / 3.0)

PRINTED = {
    "X1": {"rho_v": 0.001, "rho_l": 1.0, "W": [5.0, 6.0]},
    "X2": {"ratio_min": 940.0, "vapour_within": 0.06},
    "X4": {"nu": [0.075, 0.05, 0.02, 0.01], "d3q27_mrt": [0.00116, 0.00293, 0.0172, 0.0245],
           "d3q19_mrt": [0.00085, 0.00333, 0.0180, 0.0295], "d3q27_srt": [0.0150, 0.06542, None, None]},
    # gamma(0) and gamma(0.6) are the ends of the range quoted in Sec. III E; 0.4 and 0.8 follow from the
    # analytical capillary periods of Fig. 2c, gamma = (2 pi / T)^2 (rho_l + rho_v) / k^3, k = 2 pi / 160
    "X5": {"kappa": [0.0, 0.4, 0.6, 0.8], "gamma": [0.01034, 0.005937, 0.00395, 0.001804]},
    "X6": {"kappa": [0.0, 0.4, 0.8], "T": [7959, 10504, 19056], "T_measured": [8025, 10400, 18500]},
    "X7": {"order": 2.0},
    "X8": {"tc_over_tau": [1.9, 2.5], "paper_fit": 2.26},
}

# D3Q19 with the paper's rates (s4 = 1.2 on k220, k202, k022, s2b = 0.6) is linearly unstable at
# rest for nu <= 0.02 (FP64 oracle and GPU alike; D3Q27 is not); s4 = 1 removes the growth.
# Low-viscosity D3Q19 cases are run with STABLE_S4 and, where the paper's rates are compared,
# with those as well.
STABLE_S4 = 1.0


def params(lattice, shape, kappa=0.0, nu=None, bc=(0, 0, 0), srt=False, G_ads=0.0, s4=None, **kw):
    rates = {}
    if nu is not None:
        s = 1.0 / (3.0 * nu + 0.5)
        rates = {k: s for k in ("s0", "s1", "s2", "s2b", "s3", "s3b", "s4", "s4b", "s5", "s6")} if srt else {"s2": s}
    if s4 is not None:
        rates["s4"] = s4
    return Params(lattice=lattice, shape=shape, bc=bc, eos="piecewise", eos_p=PIECEWISE, G=-1.0, sigma=0.1,
                  kappa=kappa, G_ads=G_ads, rates=rates, **kw)


def tanh_field(dist, W=4.0):
    """liquid where dist < 0 (tanh profile of Eq. e23)"""
    return 0.5 * (RHO_L + RHO_V) - 0.5 * (RHO_L - RHO_V) * np.tanh(2.0 * dist / W)


def grid(shape):
    """x, y, z coordinate arrays shaped (nz, ny, nx)"""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def sphere(shape, R, centre=None):
    x, y, z = grid(shape)
    nx, ny, nz = shape
    cx, cy, cz = centre if centre is not None else (nx / 2.0, ny / 2.0, nz / 2.0)
    return tanh_field(np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - R)


def start(p, rho, u=None, solid=None, stream=None):
    import torch
    sim = Simulation(p, stream=stream)
    u = np.zeros((3,) + rho.shape) if u is None else u
    sim.init_fields(torch.tensor(rho, dtype=torch.float32, device="cuda"),
                    torch.tensor(u, dtype=torch.float32, device="cuda"),
                    None if solid is None else torch.tensor(solid, dtype=torch.uint8, device="cuda"))
    return sim


def pressure(sim, rho):
    """p = rho / 3 + G psi^2 / 2 (G = -1) from the library's psi."""
    psi = sim.psi(device=False).astype(np.float64)
    return rho / 3.0 - 0.5 * psi * psi


def run_all(sims, steps, chunk=2000):
    """Advance independent simulations together (one batch) by `steps` steps, checking status."""
    b = Batch(sims)
    done = 0
    try:
        while done < steps:
            n = min(chunk, steps - done)
            n += n % 2
            b.step(n)
            b.sync()
            done += n
    finally:
        b.close()
    return done


def vapour_speed(sim):
    r, u, _ = sim.moments(device=False)
    vap = r < 0.5 * (RHO_L + RHO_V)
    return float(np.sqrt((u.astype(np.float64) ** 2).sum(axis=0))[vap].mean())


# ---------------------------------------------------------------- X1 / X2
def planar_and_droplet(quick):
    out = {}
    res = {}
    for Q in (19, 27):
        nx = 100
        shape = (nx, 4, 4)
        x, _, _ = grid(shape)
        sim = start(params(Q, shape), tanh_field(np.abs(x - nx / 2 + 0.5) - nx / 4))
        run_all([sim], 4000 if quick else 20000)
        r = sim.moments(device=False)[0][0, 0].astype(np.float64)
        res[Q] = {"rho_l": float(r.max()), "rho_v": float(r.min()),
                  "W": float((r.max() - r.min()) / np.abs(np.diff(r)).max())}
        sim.close()
    out["X1"] = res
    N = 96 if quick else 200
    shape = (N, N, N)
    res = {}
    for Q in (19, 27):
        sim = start(params(Q, shape), sphere(shape, N / 4.0))
        run_all([sim], 6000 if quick else 20000)
        r = sim.moments(device=False)[0].astype(np.float64)
        rl, rv = float(r[N // 2, N // 2, N // 2]), float(r[0, 0, 0])
        res[Q] = {"N": N, "R": N / 4.0, "rho_l_centre": rl, "rho_v_far": rv, "ratio": rl / rv,
                  "vapour_dev_from_planar": abs(rv - out["X1"][Q]["rho_v"]) / out["X1"][Q]["rho_v"]}
        sim.close()
    out["X2"] = res
    return out


# ---------------------------------------------------------------- X4 spurious velocities
def spurious(quick):
    N = 80 if quick else 200
    shape = (N, N, N)
    rho = sphere(shape, N / 4.0)
    steps = 4000 if quick else 20000
    out = {}
    for nu in PRINTED["X4"]["nu"]:
        for Q, srt, s4 in ((27, False, None), (19, False, None), (19, False, STABLE_S4), (27, True, None)):
            key = f"d3q{Q}_{'srt' if srt else 'mrt'}{'' if s4 is None else '_s4_' + str(s4)}_nu{nu}"
            sim = start(params(Q, shape, nu=nu, srt=srt, s4=s4), rho)
            try:       # each case alone: an unstable one must not stop the others
                run_all([sim], steps)
                out[key] = vapour_speed(sim)
            except Exception as e:   # LBM_ERR_UNSTABLE / EOS_RANGE: the paper's NaN entries
                out[key] = "diverged: " + str(e).split(":")[0]
            sim.close()
    return {"X4": {"N": N, "steps": steps, "u_v": out}}


# ---------------------------------------------------------------- X5 Laplace
def laplace(quick, lattice=19):
    N = 96 if quick else 180
    radii = [14, 18, 22, 26] if quick else [28, 33, 38, 43, 48]
    kappas = PRINTED["X5"]["kappa"]
    shape = (N, N, N)
    steps = 6000 if quick else 20000
    gam = {}
    for kappa in kappas:
        dp = {}
        for R in radii:          # one run at a time: a diverging case does not take others along
            sim = start(params(lattice, shape, kappa=kappa), sphere(shape, R))
            try:
                run_all([sim], steps)
                rho = sim.moments(device=False)[0].astype(np.float64)
                p = pressure(sim, rho)
                dp[R] = float(p[N // 2, N // 2, N // 2] - p[0, 0, 0])
            except Exception as e:
                dp[R] = "diverged: " + str(e).split(":")[0]
            sim.close()
        ok = [R for R in radii if isinstance(dp[R], float)]
        entry = {"dp": {str(R): dp[R] for R in radii}}
        if len(ok) >= 3:
            slope, icpt = np.polyfit(np.array([2.0 / R for R in ok]), np.array([dp[R] for R in ok]), 1)
            entry.update(gamma=float(slope), intercept=float(icpt), radii_fitted=ok)
        gam[kappa] = entry
    g0 = gam.get(0.0, {}).get("gamma")
    for k, v in gam.items():
        if "gamma" in v and g0:
            v["ratio_to_kappa0"] = v["gamma"] / g0
            v["one_minus_kappa"] = 1 - k
    return {"N": N, "radii": radii, "steps": steps, "lattice": lattice,
            "by_kappa": {str(k): v for k, v in gam.items()},
            "printed_gamma": dict(zip(map(str, kappas), PRINTED["X5"]["gamma"]))}


# ---------------------------------------------------------------- X7 convergence
def convergence(quick):
    Ns = [48, 64, 96, 128] if quick else [100, 150, 200, 300]
    vals = {}
    for N in Ns:
        shape = (N, N, N)
        sim = start(params(19, shape), sphere(shape, N / 4.0))
        run_all([sim], int(4000 * N / Ns[0]) if quick else int(12000 * N / 100))
        r = sim.moments(device=False)[0].astype(np.float64)
        vals[N] = (float(r[N // 2, N // 2, N // 2]), float(r[0, 0, 0]))
        sim.close()
    ref = vals[Ns[-1]]
    err_l = {N: abs(vals[N][0] - ref[0]) for N in Ns[:-1]}
    err_v = {N: abs(vals[N][1] - ref[1]) for N in Ns[:-1]}
    order = float(-np.polyfit(np.log(Ns[:-1]), np.log([max(err_l[N], 1e-300) for N in Ns[:-1]]), 1)[0])
    return {"kappa": 0.0, "rho": {str(N): vals[N] for N in Ns}, "err_liquid": {str(N): err_l[N] for N in err_l},
            "err_vapour": {str(N): err_v[N] for N in err_v}, "order_liquid": order}


# ---------------------------------------------------------------- X6 capillary waves
def capillary(quick, gammas, nu=0.01):
    L = 80 if quick else 160
    H, D, h0 = 5 * L, 5, L / 8.0
    shape = (L, H, D)
    x, y, z = grid(shape)
    k = 2 * math.pi / L
    rho = tanh_field(y - (H / 2.0 + h0 * np.cos(k * x)))
    out = {}
    for kappa in PRINTED["X6"]["kappa"]:
        sim = start(params(19, shape, kappa=kappa, nu=nu, bc=(0, 1, 0), s4=STABLE_S4), rho)
        try:
            out[str(kappa)] = capillary_run(sim, gammas.get(kappa), k, L, H)
        except Exception as e:
            out[str(kappa)] = {"status": "diverged: " + str(e).split(":")[0]}
        sim.close()
    return {"L": L, "H": H, "D": D, "h0": h0, "nu": nu, "s4": STABLE_S4, "by_kappa": out}


def capillary_run(sim, gamma, k, L, H):
    """amplitude of the cos(kx) mode of the interface height over about two theoretical periods;
    the measured period is twice the mean spacing of its zero crossings"""
    T_theory = 2 * math.pi / math.sqrt(gamma * k ** 3 / (RHO_L + RHO_V)) if gamma else None
    horizon = int(2.3 * (T_theory or 20000))
    every = max(20, int((T_theory or 20000) / 100))
    every += every % 2
    mid = 0.5 * (RHO_L + RHO_V)
    basis = np.cos(k * np.arange(L))
    cols = np.arange(L)
    ts, amp = [], []
    t = 0
    while t < horizon:
        sim.step(every)
        t += every
        r = sim.moments(device=False, sums=False)[0].astype(np.float64).mean(axis=0)   # (ny, nx), z-averaged
        j = np.argmin(r >= mid, axis=0)           # first non-liquid row from the bottom wall, per column
        lo, hi = r[j - 1, cols], r[j, cols]
        h = (j - 1) + (lo - mid) / (lo - hi)
        amp.append(float(2.0 / L * np.dot(h - H / 2.0, basis)))
        ts.append(t)
    a = np.array(amp)
    zc = [ts[i] + (ts[i + 1] - ts[i]) * a[i] / (a[i] - a[i + 1]) for i in range(len(a) - 1) if a[i] * a[i + 1] < 0]
    T_meas = 2 * float(np.mean(np.diff(zc))) if len(zc) >= 2 else None
    return {"gamma_used": gamma, "T_theory": T_theory, "T_measured": T_meas,
            "rel_err": None if not (T_meas and T_theory) else abs(T_meas - T_theory) / T_theory,
            "zero_crossings": len(zc), "amplitude_first_last": [amp[0], amp[-1]], "status": "ok"}


# ---------------------------------------------------------------- X8 contact time
def contact_time(quick, gamma):
    """droplet (D3Q19, s4 = STABLE_S4, kappa = 0) falling at We = 10 onto a wall with G_ads = 0.23;
    contact from the first liquid cell on the wall to the start of the no-contact run that lasts
    0.6 tau (the spreading film rides on a vapour cushion for up to about half a capillary time
    before it touches again, which is not a bounce)"""
    out = {}
    for R0 in ([16] if quick else [20, 30]):
        for nu in (0.02, 0.05):
            We = 10.0
            U = math.sqrt(We * gamma / (RHO_L * R0))
            tau = math.sqrt(RHO_L * R0 ** 3 / gamma)
            L = 6 * R0
            shape = (L, L, 4 * R0)
            rho = sphere(shape, R0, centre=(L / 2.0, L / 2.0, R0 + 3.0))
            u = np.zeros((3,) + rho.shape)
            u[2] = -U * np.clip((rho - RHO_V) / (RHO_L - RHO_V), 0, 1)
            sim = start(params(19, shape, nu=nu, bc=(0, 0, 1), G_ads=0.23, s4=STABLE_S4), rho, u)
            thr = 0.5 * (RHO_L + RHO_V)
            touch = detach = zero_from = None
            t = 0
            every = 20
            hold = 0.6 * tau
            status = "ok"
            try:
                while t < 4.5 * tau and detach is None:
                    sim.step(every)
                    t += every
                    wet = sim.contact(thr)["wet"]
                    if touch is None:
                        touch = t if wet > 0 else None
                    elif wet > 0:
                        zero_from = None
                    else:
                        zero_from = t if zero_from is None else zero_from
                        if t - zero_from >= hold:
                            detach = zero_from
            except Exception as e:
                status = str(e).split(":")[0]
            sim.close()
            out[f"R0{R0}_nu{nu}"] = {"tau": tau, "U": U, "We": We, "nu": nu, "touch": touch, "detach": detach,
                                      "tc_over_tau": None if detach is None else (detach - touch) / tau,
                                      "status": status}
    return out


# ---------------------------------------------------------------- C3 full-size impact, FP32 vs FP16
def impact_fp16(quick):
    """D3Q19 impact on a neutral wall (G_ads = 0), U = 0.08, nu = 0.05, s4 = STABLE_S4, droplet two
    cells above the wall: D_f / R0 every R0 / (4 U) steps up to t* = U t / R0 = 3, both stores."""
    R0 = 12.5 if quick else 50.0
    shape = (100, 100, 50) if quick else (400, 400, 200)
    U, nu = 0.08, 0.05
    every = int(round(R0 / (4 * U)))
    every += every % 2
    n = int(3 * R0 / U / every)
    rho = sphere(shape, R0, centre=(shape[0] / 2.0, shape[1] / 2.0, R0 + 2.0))
    u = np.zeros((3,) + rho.shape)
    u[2] = -U * np.clip((rho - RHO_V) / (RHO_L - RHO_V), 0, 1)
    thr = 0.5 * (RHO_L + RHO_V)
    curves = {}
    for store in ("fp32", "fp16"):
        sim = start(params(19, shape, nu=nu, bc=(0, 0, 1), s4=STABLE_S4, store=store), rho, u)
        df = []
        for _ in range(n):
            sim.step(every)
            c = sim.contact(thr)
            df.append(0.0 if c["floor"] == 0 else 0.5 * ((c["xmax"] - c["xmin"] + 1) + (c["ymax"] - c["ymin"] + 1)))
        sim.close()
        curves[store] = df
    a, b = np.array(curves["fp32"]), np.array(curves["fp16"])
    return {"shape": shape, "R0": R0, "U": U, "nu": nu, "every": every,
            "t_star": [round(U * every * (k + 1) / R0, 3) for k in range(n)],
            "Df_over_R0_fp32": [round(v / R0, 4) for v in curves["fp32"]],
            "Df_over_R0_fp16": [round(v / R0, 4) for v in curves["fp16"]],
            "max_abs_diff_cells": float(np.abs(a - b).max())}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="smaller boxes and fewer steps")
    ap.add_argument("--cases", default="X1,X2,X4,X5,X5_27,X6,X7,X8,C3")
    a = ap.parse_args(argv)
    want = set(a.cases.split(","))
    report = {"printed": PRINTED, "quick": a.quick}
    t0 = time.time()

    def guarded(name, fn, *args):
        t = time.time()
        try:
            res = fn(*args)
        except Exception as e:   # one failing case must not hide the others
            res = {name: {"status": "failed: " + str(e)[:200]}}
        for k, v in res.items():
            report[k] = v
            print(json.dumps({k: v, "seconds": round(time.time() - t, 1)}), file=sys.stderr, flush=True)
        return res

    if want & {"X1", "X2"}:
        guarded("X1", planar_and_droplet, a.quick)
    if "X4" in want:
        guarded("X4", spurious, a.quick)
    if "X5" in want:
        guarded("X5", lambda q: {"X5": laplace(q, 19)}, a.quick)
    if "X5_27" in want:
        guarded("X5_27", lambda q: {"X5_27": laplace(q, 27)}, a.quick)
    # the printed surface tensions set the theoretical capillary periods and the impact scales
    gammas = dict(zip(PRINTED["X5"]["kappa"], PRINTED["X5"]["gamma"]))
    if "X6" in want:
        guarded("X6", lambda q: {"X6": capillary(q, gammas, 0.01)}, a.quick)
    if "X7" in want:
        guarded("X7", lambda q: {"X7": convergence(q)}, a.quick)
    if "X8" in want:
        guarded("X8", lambda q: {"X8": contact_time(q, gammas[0.0])}, a.quick)
    if "C3" in want:
        guarded("C3", lambda q: {"C3": impact_fp16(q)}, a.quick)
    report["seconds"] = time.time() - t0
    print(json.dumps(report), flush=True)
    return report


if __name__ == "__main__":
    sys.exit(0 if main() else 1)
