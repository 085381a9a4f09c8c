"""Pins for oracle/eos.py: printed spinodals, C-S critical point, Maxwell construction."""
import json
import math
import os
import warnings

import numpy as np
import pytest

import workloads
from oracle import eos

warnings.simplefilter("ignore")


def test_piecewise_spinodals_match_printed_values(golden_dir):
    pv = json.load(open(os.path.join(golden_dir, "paper_values.json")))["piecewise_eos"]
    tv, tm, tl = eos.piecewise_slopes()
    # Eq. e21 slopes
    assert tv == pytest.approx(1 / 6) and tl == pytest.approx(1 / 3) and tm == pytest.approx(-1 / 120)
    r1, r2 = eos.piecewise_spinodals(pv["rho_v"], pv["rho_l"], tv, tm, tl)
    # printed to 4 significant digits after Eq. e21
    assert round(r1, 6) == pv["rho1"]
    assert round(r2, 4) == pv["rho2"]
    # both conditions of Eq. e20 hold at the solution
    p = lambda r: eos.piecewise_pressure(r, r1, r2, tv, tm, tl)  # noqa: E731
    assert abs(p(pv["rho_l"]) - p(pv["rho_v"])) < 1e-15
    integral = tv * math.log(r1 / pv["rho_v"]) + tm * math.log(r2 / r1) + tl * math.log(pv["rho_l"] / r2)
    assert abs(integral) < 1e-14


def test_piecewise_pressure_is_continuous_with_the_three_slopes():
    tv, tm, tl = eos.piecewise_slopes()
    r1, r2 = 0.0013, 0.97
    for r in (r1, r2):
        lo, hi = eos.piecewise_pressure(r - 1e-9, r1, r2, tv, tm, tl), eos.piecewise_pressure(r + 1e-9, r1, r2, tv, tm, tl)
        assert abs(hi - lo) < 1e-9
    for (a, b, slope) in ((1e-4, 1e-3, tv), (0.1, 0.2, tm), (0.98, 1.1, tl)):
        d = (eos.piecewise_pressure(b, r1, r2, tv, tm, tl) - eos.piecewise_pressure(a, r1, r2, tv, tm, tl)) / (b - a)
        assert d == pytest.approx(slope, rel=1e-12)


def test_cs_critical_point_matches_textbook_constants():
    # Carnahan-Starling with van der Waals attraction: b rho_c = 0.52177, b R T_c / a = 0.37733
    a, b, R = 0.5, 4.0, 1.0
    rho_c, T_c = eos.cs_critical_point(a, b, R)
    assert b * rho_c == pytest.approx(0.52177, abs=2e-5)
    assert b * R * T_c / a == pytest.approx(0.37733, abs=2e-5)


def _mu_closed_form(rho, a, b, R, T):
    # chemical potential of the C-S fluid: ideal + hard-sphere excess + mean-field attraction
    eta = b * rho / 4.0
    return R * T * (math.log(rho) + (8 * eta - 9 * eta ** 2 + 3 * eta ** 3) / (1 - eta) ** 3) - 2 * a * rho


@pytest.mark.parametrize("frac", [0.5, 0.7, 0.9])
def test_cs_maxwell_construction(frac):
    a, b, R = 0.5, 4.0, 1.0
    _, T_c = eos.cs_critical_point(a, b, R)
    T = frac * T_c
    rv, rl = eos.cs_maxwell(a, b, R, T)
    p_v, p_l = eos.cs_pressure(rv, a, b, R, T), eos.cs_pressure(rl, a, b, R, T)
    assert abs(p_v - p_l) < 1e-13
    # closed-form chemical potentials agree (independent of the quadrature used by the oracle)
    assert abs(_mu_closed_form(rv, a, b, R, T) - _mu_closed_form(rl, a, b, R, T)) < 1e-11
    # equal areas in the specific volume: integral of (p(v) - p_coex) dv over [v_l, v_v] vanishes
    v = np.geomspace(1 / rl, 1 / rv, 400001)
    dv = np.diff(v)
    pv = eos.cs_pressure(1 / v, a, b, R, T) - p_v
    area = float(np.sum(0.5 * (pv[1:] + pv[:-1]) * dv))
    scale = float(np.sum(np.abs(0.5 * (pv[1:] + pv[:-1])) * dv))
    assert abs(area) < 1e-6 * scale


def test_stored_constants_are_the_oracle_values():
    c = workloads.constants()
    a, b, R = c["cs"]["a"], c["cs"]["b"], c["cs"]["R"]
    rho_c, T_c = eos.cs_critical_point(a, b, R)
    assert c["cs"]["T_c"] == pytest.approx(T_c, rel=1e-12)
    for frac in (0.7, 0.5):
        d = c["cs"][f"T{frac}"]
        rv, rl = eos.cs_maxwell(a, b, R, d["T"])
        assert d["rho_v"] == pytest.approx(rv, rel=1e-10) and d["rho_l"] == pytest.approx(rl, rel=1e-10)
    pw = c["piecewise"]
    r1, r2 = eos.piecewise_spinodals(pw["rho_v"], pw["rho_l"], pw["theta_v"], pw["theta_m"], pw["theta_l"])
    assert pw["rho1"] == pytest.approx(r1, rel=1e-12) and pw["rho2"] == pytest.approx(r2, rel=1e-12)


def test_bulk_pressure_equals_eos_pressure():
    # Eq. e16 with the square-root psi of Sec. II C returns p_EOS
    a, b, R, T = 0.5, 4.0, 1.0, 0.03
    rho = np.linspace(0.001, 0.45, 50)
    p = eos.cs_pressure(rho, a, b, R, T)
    psi = np.sqrt(eos.psi_squared(p, rho, -1.0))
    assert np.allclose(eos.bulk_pressure(rho, psi, -1.0), p, rtol=0, atol=1e-15)
