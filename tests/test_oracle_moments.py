"""Pins for oracle/moments.py against what the paper prints and the algebra fixes."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import lattice as la
from oracle import moments as mo
from oracle import velocity_space as vs


def _printed(golden_dir, name):
    rows = [r for r in open(os.path.join(golden_dir, name)) if not r.startswith("#")]
    return [[int(v) for v in r.split()] for r in rows]


@pytest.mark.parametrize("Q,name", [(27, "M27_printed.txt"), (19, "M19_printed.txt")])
def test_M_equals_printed_matrix(golden_dir, Q, name):
    # M is rebuilt from the moment definitions of Eq. e11 and must equal the printed matrix
    assert mo.matrix_exact(Q) == _printed(golden_dir, name)


def test_nonzero_counts_match_table_I(golden_dir):
    t = json.load(open(os.path.join(golden_dir, "paper_values.json")))["table1_nonzeros"]
    for Q in (27, 19):
        M, Mi = mo.matrices_exact(Q)
        assert sum(v != 0 for r in M for v in r) == t[f"M{Q}"]
        assert sum(v != 0 for r in Mi for v in r) == t[f"Minv{Q}"]


@pytest.mark.parametrize("Q", [19, 27])
def test_inverse_is_exact(Q):
    M, Mi = mo.matrices_exact(Q)
    for i in range(Q):
        for j in range(Q):
            assert sum(Fraction(M[i][k]) * Mi[k][j] for k in range(Q)) == (1 if i == j else 0)
    # float copies agree with the exact ones
    Mf, Mif = mo.matrices(Q)
    assert np.abs(Mf @ Mif - np.eye(Q)).max() < 1e-14


def test_d3q19_inverse_is_extracted_from_d3q27():
    # App. C: the D3Q19 M^-1 equals the D3Q27 M^-1 restricted to the first 19 velocities and
    # the 19 retained moments
    _, Mi27 = mo.matrices_exact(27)
    _, Mi19 = mo.matrices_exact(19)
    for i in range(19):
        for c, k in enumerate(mo.D3Q19_MOMENTS):
            assert Mi19[i][c] == Mi27[i][k]


def test_relaxation_vector_matches_eq_e12(golden_dir):
    pv = json.load(open(os.path.join(golden_dir, "paper_values.json")))
    rates = {k: float(10 + n) for n, k in enumerate(mo.RATE_NAMES)}
    for Q, key in ((27, "relaxation_diag_27"), (19, "relaxation_diag_19")):
        want = [rates[r] for r in pv[key]["rates"]]
        assert list(mo.relaxation_vector(Q, rates)) == want
    d = pv["default_rates"]
    for k, v in mo.DEFAULT_RATES.items():
        assert v == d.get(k, d["others"])


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.3, 1.5, n), rng.uniform(-0.15, 0.15, (3, n)), rng.uniform(-0.1, 0.1, (3, n))


def test_equilibrium_moments_are_moments_of_hermite_feq():
    # D3Q27: m^eq of Eq. e13 = M f^eq with f^eq of Eq. e5 (with the 1/2 on the quadratic term)
    rho, u, _ = _rand(50, 1)
    M, _ = mo.matrices(27)
    assert np.abs(M @ vs.feq_hermite(27, rho, u) - mo.equilibrium(27, rho, *u)).max() < 1e-14
    # as printed (no 1/2) it does not reproduce Eq. e13: the reading is needed
    assert np.abs(M @ vs.feq_as_printed(27, rho, u) - mo.equilibrium(27, rho, *u)).max() > 1e-3


def test_forcing_moments_are_moments_of_guo_force():
    # D3Q27: F~ of Eq. e14 = M F_bar with F_bar of Eq. e6
    _, u, F = _rand(50, 2)
    M, _ = mo.matrices(27)
    assert np.abs(M @ vs.guo_force(27, u, F) - mo.forcing(27, *F, *u)).max() < 1e-15


def test_forcing_is_derivative_of_equilibrium():
    # F~ = d m^eq / d(rho u) . F at fixed rho (a second, independent form of Eq. e14)
    rho, u, F = _rand(20, 3)
    h = 1e-6
    for Q in (19, 27):
        d = np.zeros((Q, rho.size))
        for a in range(3):
            up, um = u.copy(), u.copy()
            up[a] += h / rho
            um[a] -= h / rho
            d += (mo.equilibrium(Q, rho, *up) - mo.equilibrium(Q, rho, *um)) / (2 * h) * F[a]
        assert np.abs(d - mo.forcing(Q, *F, *u)).max() < 1e-8


def test_equilibrium_returns_rho_and_momentum():
    rho, u, _ = _rand(10, 4)
    for Q in (19, 27):
        m = mo.equilibrium(Q, rho, *u)
        assert np.allclose(m[0], rho) and np.allclose(m[1:4], rho * u)
        _, Minv = mo.matrices(Q)
        f = Minv @ m
        e = la.velocities(Q)
        assert np.allclose(f.sum(0), rho, rtol=1e-14)
        assert np.allclose(e.T @ f, rho * u, atol=1e-15)


def test_d3q19_extracted_equilibrium_differs_only_in_fourth_order_rows():
    # The D3Q19 m^eq of App. C is the D3Q27 vector restricted.  Against the moments of the
    # standard D3Q19 Hermite equilibrium it agrees up to second order (rows 0..9) and in the
    # third-order rows; rows k220, k202, k022 differ by -rho u_z^2/6, -rho u_y^2/6, -rho u_x^2/6.
    rho, u, _ = _rand(30, 5)
    M, _ = mo.matrices(19)
    m_h = M @ vs.feq_hermite(19, rho, u)
    m_p = mo.equilibrium(19, rho, *u)
    assert np.abs(m_h[:16] - m_p[:16]).max() < 1e-15
    diff = m_h[16:] - m_p[16:]
    expect = -rho * np.stack([u[2] ** 2, u[1] ** 2, u[0] ** 2]) / 6.0
    assert np.abs(diff - expect).max() < 1e-15
