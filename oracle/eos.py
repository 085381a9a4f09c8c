"""Equations of state and the square-root pseudopotential (oracle; test infrastructure only).

* Carnahan-Starling (C-S) EOS, named in Sec. III A.  The paper does not print
  its formula; the standard C-S form with a van der Waals attraction is used:
  p = rho R T (1 + eta + eta^2 - eta^3) / (1 - eta)^3 - a rho^2, eta = b rho / 4.
* Piecewise-linear EOS, Eq. e19, with slopes of Eq. e21 and the spinodal
  densities rho_1, rho_2 from the two equilibrium conditions of Eq. e20 (read as
  p(rho_l) - p(rho_v) = 0 and the integral of dp / rho from rho_v to rho_l = 0;
  the leading integral sign on the first line is a typesetting slip).
* psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2)), Sec. II C, with c = 1.
* bulk pressure p = rho c_s^2 + G c^2 psi^2 / 2, Eq. e16.

Pins (tests/test_oracle_eos.py): rho_1 = 0.001325 and rho_2 = 0.9758 printed in
Sec. III A for rho_v = 0.001, rho_l = 1; the C-S critical point against the
textbook reduced constants (b rho_c = 0.5218, b R T_c / a = 0.3773); the
Maxwell construction checked by an independent equal-area quadrature in the
specific volume; p of Eq. e16 equal to p_EOS by construction.
"""
import math

import numpy as np
from scipy import integrate, optimize

CS2 = 1.0 / 3.0


# ---------------------------------------------------------------- Carnahan-Starling
def cs_pressure(rho, a, b, R, T):
    eta = b * rho / 4.0
    return rho * R * T * (1.0 + eta + eta * eta - eta ** 3) / (1.0 - eta) ** 3 - a * rho * rho


def cs_dpdrho(rho, a, b, R, T):
    """Analytic derivative of cs_pressure with respect to rho."""
    eta = b * rho / 4.0
    g = (1.0 + eta + eta * eta - eta ** 3) / (1.0 - eta) ** 3
    dg = ((1.0 + 2.0 * eta - 3.0 * eta * eta) * (1.0 - eta) + 3.0 * (1.0 + eta + eta * eta - eta ** 3)) \
        / (1.0 - eta) ** 4
    return R * T * (g + eta * dg) - 2.0 * a * rho


def cs_critical_point(a, b, R):
    """(rho_c, T_c): where dp/drho and d2p/drho2 vanish together."""
    def d2(rho, T, h=1e-6):
        return (cs_dpdrho(rho + h, a, b, R, T) - cs_dpdrho(rho - h, a, b, R, T)) / (2 * h)

    def eqs(v):
        rho, T = v
        return [cs_dpdrho(rho, a, b, R, T), d2(rho, T)]

    # crude starting point (order of magnitude only): eta ~ 1/8, R T ~ a / (3 b)
    rho_c, T_c = optimize.fsolve(eqs, [0.5 / b, a / (3.0 * b * R)], xtol=1e-14)
    return float(rho_c), float(T_c)


def cs_maxwell(a, b, R, T):
    """Coexistence densities (rho_v, rho_l) at temperature T < T_c: equal pressure and
    equal chemical potential, mu(rho_l) - mu(rho_v) = integral of (dp/drho)/rho."""
    rho_c, T_c = cs_critical_point(a, b, R)
    if not T < T_c:
        raise ValueError("T must be below the critical temperature")

    # spinodals bracket the two branches
    lo = optimize.brentq(lambda r: cs_dpdrho(r, a, b, R, T), 1e-12, rho_c)
    hi = optimize.brentq(lambda r: cs_dpdrho(r, a, b, R, T), rho_c, 0.99 * 4.0 / b)

    def dmu(r1, r2):
        val, _ = integrate.quad(lambda r: cs_dpdrho(r, a, b, R, T) / r, r1, r2,
                                epsabs=1e-14, epsrel=1e-12, limit=400)
        return val

    p_lo = cs_pressure(hi, a, b, R, T)   # pressure at the liquid-side spinodal (local minimum)
    p_hi = cs_pressure(lo, a, b, R, T)   # pressure at the vapour-side spinodal (local maximum)
    rho_max = 0.999 * 4.0 / b

    def branches(P):
        rv = optimize.brentq(lambda r: cs_pressure(r, a, b, R, T) - P, 1e-300, lo, xtol=1e-300, rtol=1e-15)
        rl = optimize.brentq(lambda r: cs_pressure(r, a, b, R, T) - P, hi, rho_max, xtol=1e-300, rtol=1e-15)
        return rv, rl

    # equal pressure by construction of the branches; equal chemical potential picks P
    P_min = p_lo * (1 + 1e-12) if p_lo > 0 else 1e-30 * p_hi
    Pc = optimize.brentq(lambda P: dmu(*branches(P)), P_min, p_hi * (1 - 1e-12), xtol=1e-300, rtol=1e-15)
    rv, rl = branches(Pc)
    if not (0 < rv < lo < hi < rl):
        raise RuntimeError("Maxwell construction converged to a spurious root")
    return rv, rl


# ---------------------------------------------------------------- piecewise linear (Eq. e19)
def piecewise_pressure(rho, rho1, rho2, theta_v, theta_m, theta_l):
    rho = np.asarray(rho, dtype=np.float64)
    p1 = rho1 * theta_v
    p2 = p1 + (rho2 - rho1) * theta_m
    return np.where(rho <= rho1, rho * theta_v,
                    np.where(rho <= rho2, p1 + (rho - rho1) * theta_m, p2 + (rho - rho2) * theta_l))


def piecewise_slopes():
    """Eq. e21: theta_v = c_s^2 / 2, theta_l = c_s^2, theta_m = -c_s^2 / 40."""
    return CS2 / 2.0, -CS2 / 40.0, CS2


def piecewise_spinodals(rho_v, rho_l, theta_v, theta_m, theta_l):
    """Solve Eq. e20 for (rho_1, rho_2).

    Mechanical equilibrium (p(rho_l) = p(rho_v)) is linear in rho_1, rho_2 and gives
    rho_2 as a function of rho_1; the chemical condition is then a scalar root in rho_1.
    """
    def rho2_of(r1):
        # (r1 - rv) tv + (r2 - r1) tm + (rl - r2) tl = 0
        return (rho_v * theta_v - rho_l * theta_l - r1 * (theta_v - theta_m)) / (theta_m - theta_l)

    def chem(r1):
        r2 = rho2_of(r1)
        return (math.log(r1 / rho_v) * theta_v + math.log(r2 / r1) * theta_m
                + math.log(rho_l / r2) * theta_l)

    # rho_1 lies between rho_v and the value that puts rho_2 at rho_l
    r1_hi = (rho_v * theta_v - rho_l * theta_l - rho_l * (theta_m - theta_l)) / (theta_v - theta_m)
    r1 = optimize.brentq(chem, rho_v * (1 + 1e-12), r1_hi * (1 - 1e-12), xtol=1e-16, rtol=1e-15)
    return r1, rho2_of(r1)


# ---------------------------------------------------------------- pseudopotential
def psi_squared(p_eos, rho, G):
    """psi^2 = 2 (p_EOS - rho c_s^2) / (G c^2) with c = 1 (Sec. II C)."""
    return 2.0 * (p_eos - rho * CS2) / G


def bulk_pressure(rho, psi, G):
    """Eq. e16 with c = 1."""
    return rho * CS2 + 0.5 * G * psi * psi
