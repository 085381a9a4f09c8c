"""Pins for oracle/lbm.py that the algebra of the step fixes exactly (small boxes)."""
import numpy as np
import pytest

import workloads as W
from oracle import lbm
from oracle import moments as mo
from oracle import velocity_space as vs

CS = W.constants()["cs"]


def _cs_params(Q, shape, T_key="T0.7", **kw):
    t = CS[T_key]
    return lbm.Params(lattice=Q, shape=shape, eos="cs", eos_p=(CS["a"], CS["b"], CS["R"], t["T"]),
                      G=-1.0, sigma=0.1, **kw)


def _droplet_state(Q, shape, R, **kw):
    t = CS["T0.7"]
    rho, u = W.droplet(shape, R, t["rho_l"], t["rho_v"])
    rng = np.random.default_rng(7)
    u = u + 0.01 * rng.standard_normal(u.shape)
    return lbm.State.from_fields(_cs_params(Q, shape, **kw), rho, u)


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("multiphase", [False, True])
def test_rest_state_is_a_fixed_point(Q, multiphase):
    shape = (6, 5, 4)
    if multiphase:
        p = _cs_params(Q, shape, kappa=0.5)
        rho0 = CS["T0.7"]["rho_l"]
    else:
        p = lbm.Params(lattice=Q, shape=shape)
        rho0 = 1.0
    s = lbm.State.from_fields(p, np.full((4, 5, 6), rho0), np.zeros((3, 4, 5, 6)))
    f0 = s.f.copy()
    s.run(5)
    assert np.abs(s.f - f0).max() < 1e-15 * rho0 * 10


@pytest.mark.parametrize("Q", [19, 27])
def test_mass_and_momentum_conserved_on_periodic_box(Q):
    # F_int is pairwise antisymmetric and Eq. e17 only touches m_4..m_9, so total mass and
    # total momentum (sum f e + F/2) are invariants of the periodic multiphase step
    s = _droplet_state(Q, (12, 10, 8), 3.0, kappa=0.6)
    m0 = s.sums()
    s.run(20)
    m1 = s.sums()
    assert abs(m1[0] - m0[0]) < 1e-13 * m0[0]
    assert np.abs(m1[1:] - m0[1:]).max() < 1e-14 * m0[0]
    # ... and the step is not trivial
    assert np.abs(s.moments()[1]).max() > 1e-3


@pytest.mark.parametrize("Q", [19, 27])
def test_result_independent_of_s0_s1(Q):
    a = _droplet_state(Q, (8, 8, 8), 2.5, kappa=0.3)
    b = _droplet_state(Q, (8, 8, 8), 2.5, kappa=0.3)
    b.p.rates.update(s0=0.4, s1=1.7)
    a.run(3)
    b.run(3)
    assert np.abs(a.f - b.f).max() < 1e-14


def test_srt_d3q27_equals_velocity_space_bgk_with_guo_forcing():
    # All rates equal: the non-orthogonal MRT reduces to SRT (Sec. II B).  For D3Q27 the
    # moment-space step must equal BGK + Guo forcing written without any transform.
    tau = 0.8
    shape = (8, 7, 6)
    s_m = _droplet_state(27, shape, 2.5)
    s_m.p.rates = {k: 1.0 / tau for k in mo.RATE_NAMES}
    s_m.p.sigma = 0.0
    s_m.p.g = (1e-5, -2e-5, 3e-5)
    s_v = lbm.State(s_m.p, s_m.f.copy(), s_m.solid.copy())
    for _ in range(3):
        s_m.step()
        vs.step_with(s_v, lambda f, rho, u, F, forces, psi: vs.bgk_guo_collide(f, rho, u, F, tau, 27))
    assert np.abs(s_m.f - s_v.f).max() < 1e-14


@pytest.mark.parametrize("Q", [19, 27])
def test_moment_space_equals_dense_lambda_form(Q):
    # Eq. e8 in moment space against Eq. e7 with Lambda = M^-1 S M, all multiphase terms on,
    # walls on z with a wetting force and random solid cells
    shape = (8, 7, 6)
    rng = np.random.default_rng(3)
    t = CS["T0.7"]
    rho = t["rho_v"] + (t["rho_l"] - t["rho_v"]) * rng.uniform(0.0, 1.0, (6, 7, 8))
    u = 0.02 * rng.standard_normal((3, 6, 7, 8))
    solid = W.random_mask(shape, 0.1, seed=11).astype(bool)
    p = _cs_params(Q, shape, kappa=0.4, G_ads=0.2, bc=(0, 0, 1), g=(0.0, 0.0, -1e-5))
    p.rates.update(s3=1.1, s4=1.3, s5=1.4, s6=0.9, s4b=1.05)
    s_m = lbm.State.from_fields(p, rho, u, solid)
    s_v = lbm.State(p, s_m.f.copy(), s_m.solid.copy())
    for _ in range(2):
        s_m.step()
        vs.step_with(s_v, lambda f, rho_, u_, F, forces, psi: vs.lambda_collide(f, rho_, u_, F, forces, psi, p))
    assert np.abs(s_m.f - s_v.f).max() < 1e-13


@pytest.mark.parametrize("Q", [19, 27])
def test_mass_conserved_in_closed_box_with_solids(Q):
    shape = (7, 6, 5)
    rng = np.random.default_rng(5)
    rho = 1.0 + 0.05 * rng.standard_normal((5, 6, 7))
    u = 0.03 * rng.standard_normal((3, 5, 6, 7))
    solid = W.random_mask(shape, 0.15, seed=2).astype(bool)
    p = lbm.Params(lattice=Q, shape=shape, bc=(1, 1, 1))
    s = lbm.State.from_fields(p, rho, u, solid)
    m0 = s.sums()[0]
    s.run(30)
    assert abs(s.sums()[0] - m0) < 1e-13 * m0


@pytest.mark.parametrize("Q", [19, 27])
def test_neutral_wall_fixed_point_and_wetting_sign(Q):
    # G_ads = 0: uniform fluid next to a wall feels no net force (neutral wall, Sec. III E).
    shape = (4, 4, 6)
    rho0 = CS["T0.7"]["rho_l"]
    p = _cs_params(Q, shape, bc=(0, 0, 1), kappa=0.5)
    s = lbm.State.from_fields(p, np.full((6, 4, 4), rho0), np.zeros((3, 6, 4, 4)))
    f0 = s.f.copy()
    s.run(3)
    assert np.abs(s.f - f0).max() < 1e-15
    # G_ads > 0 pushes fluid away from the walls (hydrophobic), G_ads < 0 pulls it in
    for G_ads, sign in ((0.2, 1.0), (-0.2, -1.0)):
        p2 = _cs_params(Q, shape, bc=(0, 0, 1), G_ads=G_ads)
        s2 = lbm.State.from_fields(p2, np.full((6, 4, 4), rho0), np.zeros((3, 6, 4, 4)))
        _, _, forces, _, _ = s2.fields()
        Fz = forces["F_ads"][2]
        assert np.all(sign * Fz[0] > 0) and np.all(sign * Fz[-1] < 0)
        assert np.abs(Fz[1:-1]).max() == 0.0


def test_equilibrium_initialisation_reproduces_fields():
    shape = (6, 5, 4)
    rho, u = W.perturbed(shape, seed=1)
    for Q in (19, 27):
        s = lbm.State.from_fields(lbm.Params(lattice=Q, shape=shape), rho, u)
        r, uu = s.moments()
        assert np.abs(r - rho).max() < 1e-15 and np.abs(uu - u).max() < 1e-15


def test_psi_out_of_range_aborts():
    shape = (4, 4, 4)
    p = _cs_params(19, shape)
    rho = np.full((4, 4, 4), 0.7)   # beyond the C-S range where psi^2 >= 0
    with pytest.raises(FloatingPointError):
        lbm.State.from_fields(p, rho, np.zeros((3, 4, 4, 4))).step()
