"""Physics pins for the oracle: closed forms and values the paper states (a few seconds each)."""
import json
import os

import numpy as np
import pytest
from scipy.optimize import curve_fit

import workloads as W
from oracle import eos, lbm
from oracle import moments as mo


def _rates(**kw):
    r = dict(mo.DEFAULT_RATES)
    r.update(kw)
    return r


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("s2", [1.2, 1.7])
def test_shear_wave_decays_at_the_viscosity_set_by_s2(Q, s2):
    # nu = (1/s2 - 1/2) c_s^2 (text after Eq. e12; Eq. ea12): u_x = U sin(kz) decays as exp(-nu k^2 t)
    L = 32
    p = lbm.Params(lattice=Q, shape=(1, 1, L), rates=_rates(s2=s2))
    s = lbm.State.from_fields(p, *W.shear_wave((1, 1, L), 1e-3))
    a0 = np.abs(s.moments()[1][0]).max()
    s.run(300)
    a1 = np.abs(s.moments()[1][0]).max()
    nu, k = (1 / s2 - 0.5) / 3, 2 * np.pi / L
    assert -np.log(a1 / a0) / 300 == pytest.approx(nu * k * k, rel=0.02)


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("s2b", [0.6, 1.5])
def test_sound_wave_attenuation_sets_bulk_viscosity(Q, s2b):
    # xi = 2/3 (1/s2b - 1/2) c_s^2 (text after Eq. e12): a standing sound wave decays at
    # (2/3 nu + xi/2) k^2 and oscillates at c_s k
    L = 32
    rates = _rates(s2b=s2b)
    p = lbm.Params(lattice=Q, shape=(L, 1, 1), rates=rates)
    x = np.arange(L)
    rho = (1 + 1e-4 * np.cos(2 * np.pi * x / L)).reshape(1, 1, L)
    s = lbm.State.from_fields(p, rho, np.zeros((3, 1, 1, L)))
    amps = []
    for _ in range(300):
        amps.append(np.dot(s.moments()[0][0, 0] - 1, np.cos(2 * np.pi * x / L)) * 2 / L)
        s.step()
    t = np.arange(300)
    k = 2 * np.pi / L
    (A, g, w), _ = curve_fit(lambda t, A, g, w: A * np.exp(-g * t) * np.cos(w * t), t, np.array(amps),
                             p0=[1e-4, 1e-3, k / np.sqrt(3)])
    nu, xi = (1 / rates["s2"] - 0.5) / 3, 2 / 3 * (1 / s2b - 0.5) / 3
    assert g == pytest.approx((2 / 3 * nu + xi / 2) * k * k, rel=0.03)
    assert w == pytest.approx(k / np.sqrt(3), rel=0.005)


@pytest.mark.parametrize("Q", [19, 27])
def test_poiseuille_between_bounce_back_walls(Q):
    # walls half-way outside planes 0 and H-1; body force g: u = g/(2 nu) (z + 1/2)(H - 1/2 - z)
    H, g, s2 = 16, 1e-6, 0.8
    p = lbm.Params(lattice=Q, shape=(1, 1, H), bc=(0, 0, 1), rates=_rates(s2=s2), g=(g, 0.0, 0.0))
    s = lbm.State.from_fields(p, np.ones((H, 1, 1)), np.zeros((3, H, 1, 1)))
    s.run(2500)
    nu, z = (1 / s2 - 0.5) / 3, np.arange(H)
    ua = g / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
    un = s.moments()[1][0, :, 0, 0]
    assert np.abs(un - ua).max() < 0.01 * ua.max()


@pytest.mark.parametrize("Q", [19, 27])
def test_planar_coexistence_and_interface_width(golden_dir, Q):
    # Sec. III A: piecewise EOS (Eqs. e19-e21), sigma = 0.1, G = -1: planar interfaces reproduce
    # rho_v = 0.001 and rho_l = 1, and the width of Eq. e23 lies in 5 <= W <= 6.
    pv = json.load(open(os.path.join(golden_dir, "paper_values.json")))
    c = W.constants()["piecewise"]
    pe = (c["rho1"], c["rho2"], c["theta_v"], c["theta_m"], c["theta_l"])
    p = lbm.Params(lattice=Q, shape=(100, 1, 1), eos="piecewise", eos_p=pe,
                   G=pv["piecewise_eos"]["G"], sigma=pv["piecewise_eos"]["sigma"])
    s = lbm.State.from_fields(p, *W.slab((100, 1, 1), 50, 1.0, 0.001, W=4.0))
    s.run(4000)
    r = s.moments()[0][0, 0]
    assert r.max() == pytest.approx(pv["piecewise_eos"]["rho_l"], rel=0.005)
    assert r.min() == pytest.approx(pv["piecewise_eos"]["rho_v"], rel=0.05)
    width = (r.max() - r.min()) / np.abs(np.diff(r)).max()
    assert pv["interface_width"]["W_min"] <= width <= pv["interface_width"]["W_max"]


def _laplace(R, kappa):
    c = W.constants()["cs"]
    t = c["T0.7"]
    shape = (48, 48, 1)
    p = lbm.Params(lattice=19, shape=shape, eos="cs", eos_p=(c["a"], c["b"], c["R"], t["T"]),
                   G=-1.0, sigma=0.1, kappa=kappa)
    s = lbm.State.from_fields(p, *W.cylinder_droplet(shape, R, t["rho_l"], t["rho_v"]))
    s.run(1000)
    r = s.moments()[0][0]
    pin = eos.cs_pressure(r[24, 24], c["a"], c["b"], c["R"], t["T"])
    pout = eos.cs_pressure(r[0, 0], c["a"], c["b"], c["R"], t["T"])
    return pin - pout


def test_laplace_law_and_surface_tension_scaling():
    # Sec. III C: dp = gamma * (curvature); for a liquid column dp = gamma / R, so dp * R is the
    # same for every radius; Eq. ea18: gamma is proportional to (1 - kappa)
    g = {}
    for kappa in (0.0, 0.5):
        d8, d12 = _laplace(8, kappa), _laplace(12, kappa)
        assert d8 > d12 > 0
        assert d8 * 8 == pytest.approx(d12 * 12, rel=0.02)
        g[kappa] = 0.5 * (d8 * 8 + d12 * 12)
    assert g[0.5] / g[0.0] == pytest.approx(0.5, abs=0.05)


@pytest.mark.parametrize("Q", [19, 27])
def test_variable_viscosity_sets_the_local_shear_rate(Q):
    # Sec. IV A: nu(rho) = nu_v + (nu_l - nu_v)(rho - rho_v)/(rho_l - rho_v), each cell relaxing its
    # shear moments at the s_nu that nu = (1/s_nu - 1/2) c_s^2 (text after Eq. e12) gives.  A shear wave
    # in a uniform fluid of density rho0 then decays at nu(rho0) k^2.  Three densities: both ends of the
    # interpolation (a swapped nu_l / nu_v fails) and one a quarter of the way (a non-linear or
    # mis-anchored interpolation fails); the expected nu is written out from the stated numbers.
    L = 64
    rho_v, rho_l, nu_v, nu_l = 0.5, 1.5, 0.02, 0.2
    k = 2 * np.pi / L
    for rho0, nu in ((0.5, 0.02), (1.5, 0.2), (0.75, 0.065)):
        p = lbm.Params(lattice=Q, shape=(1, 1, L), variable_nu=True, nu_l=nu_l, nu_v=nu_v,
                       rho_l=rho_l, rho_v=rho_v)
        s = lbm.State.from_fields(p, *W.shear_wave((1, 1, L), 1e-3, rho0=rho0))
        a0 = np.abs(s.moments()[1][0]).max()
        s.run(400)
        a1 = np.abs(s.moments()[1][0]).max()
        assert -np.log(a1 / a0) / 400 == pytest.approx(nu * k * k, rel=0.02), (rho0, nu)
    # the rate itself, cell by cell, on a field spanning the range: 1 / (3 nu + 1/2)
    p = lbm.Params(lattice=Q, variable_nu=True, nu_l=nu_l, nu_v=nu_v, rho_l=rho_l, rho_v=rho_v)
    rho = np.array([0.5, 0.75, 1.0, 1.5])
    assert np.allclose(lbm.shear_rate(rho, p), [1 / 0.56, 1 / 0.695, 1 / 0.83, 1 / 1.1], rtol=1e-14, atol=0)


@pytest.mark.parametrize("Q", [19, 27])
def test_adsorption_force_magnitude_at_flat_walls(Q):
    # Sec. III E: F_ads = -G_ads psi(x) sum_i w_i psi(x) s(x + e_i) e_i.  For a uniform fluid next to a
    # flat wall the solid neighbours of a first-plane cell are the links with e_z = -1, whose weights
    # add up to 1/2 on either lattice (D3Q19: 1/6 + 4/12; D3Q27: 2/9 + 4/18 + 4/72), so
    # F_ads = (0, 0, +G_ads psi^2 / 2) at the bottom plane and -G_ads psi^2 / 2 at the top one.  On the
    # edge where a y wall meets the z wall the solid links are those with e_y = -1 or e_z = -1: the z sum
    # takes 1/2 from e_z = -1 and loses the links (e_y = -1, e_z = +1), 1/12 on either lattice (D3Q19:
    # one edge link; D3Q27: 1/18 + 2/72), so F_z = 5/12 G_ads psi^2, and F_y likewise.  psi^2 is the
    # square-root pseudopotential of Sec. II C, 2 (p_EOS - rho c_s^2) / G, with the C-S pressure.
    t = W.constants()["cs"]["T0.7"]
    c = W.constants()["cs"]
    rho0, G, G_ads = 0.3, -1.0, 0.17
    psi2 = 2.0 * (eos.cs_pressure(rho0, c["a"], c["b"], c["R"], t["T"]) - rho0 / 3.0) / G
    assert 0.0 < psi2 < 0.5                  # psi^2 != psi: a wrong power of psi fails
    shape = (4, 5, 6)
    p = lbm.Params(lattice=Q, shape=shape, bc=(0, 0, 1), eos="cs", eos_p=(c["a"], c["b"], c["R"], t["T"]),
                   G=G, G_ads=G_ads)
    s = lbm.State.from_fields(p, np.full((6, 5, 4), rho0), np.zeros((3, 6, 5, 4)))
    F = s.fields()[2]["F_ads"]
    assert np.allclose(F[2][0], 0.5 * G_ads * psi2, rtol=1e-13, atol=0)
    assert np.allclose(F[2][-1], -0.5 * G_ads * psi2, rtol=1e-13, atol=0)
    assert np.abs(F[:2]).max() < 1e-17 and np.abs(F[2][1:-1]).max() == 0.0
    p.bc = (0, 1, 1)
    s = lbm.State.from_fields(p, np.full((6, 5, 4), rho0), np.zeros((3, 6, 5, 4)))
    F = s.fields()[2]["F_ads"]
    assert np.allclose(F[1][0, 0], 5.0 / 12.0 * G_ads * psi2, rtol=1e-13, atol=0)   # bottom-front edge
    assert np.allclose(F[2][0, 0], 5.0 / 12.0 * G_ads * psi2, rtol=1e-13, atol=0)
    assert np.allclose(F[2][0, 1:-1], 0.5 * G_ads * psi2, rtol=1e-13, atol=0)   # away from the edge
