"""Independent velocity-space forms of the collision (oracle; test infrastructure only).

Two second forms of the same step, used only to pin ``lbm.collide``:

* ``bgk_guo_collide``: single-relaxation-time BGK with Guo forcing written in
  velocity space with no transform at all: f^eq of Eq. e5 and F_bar of Eq. e6.
  With every rate of S equal to 1/tau the non-orthogonal MRT reduces to SRT
  (Sec. II B), so for D3Q27 this must equal ``lbm.collide`` when the Eq. e17
  modifications are off (sigma = kappa = 0).
* ``lambda_collide``: Eq. e7 with the dense Q x Q collision matrix
  Lambda = M^-1 S M, f^eq = M^-1 m^eq and F_bar' = M^-1 F~' (including Eq. e17);
  this is the velocity-space statement the moment-space Eq. e8 was derived from.

Eq. e5 as printed has no factor 1/2 on the quadratic term; with that factor M f^eq
reproduces Eq. e13 exactly for D3Q27, without it it does not (tests pin this), so
the factor is included here.
"""
import numpy as np

from . import lbm as _lbm
from . import moments as _mom
from .lattice import omega, velocities

CS2 = _lbm.CS2


def feq_hermite(Q, rho, u):
    """Eq. e5 with the 1/2 on the quadratic term: rho omega_i [1 + e.u/cs2 + (e.u)^2/(2 cs4) - u.u/(2 cs2)]."""
    e = velocities(Q).astype(np.float64)
    w = omega(Q)
    eu = np.tensordot(e, u, axes=(1, 0))
    uu = (u * u).sum(axis=0)
    return w.reshape((Q,) + (1,) * rho.ndim) * rho[None] * (
        1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu[None] / (2.0 * CS2))


def feq_as_printed(Q, rho, u):
    """Eq. e5 exactly as printed (no 1/2 on the quadratic term); used only to show the reading."""
    e = velocities(Q).astype(np.float64)
    w = omega(Q)
    eu = np.tensordot(e, u, axes=(1, 0))
    uu = (u * u).sum(axis=0)
    return w.reshape((Q,) + (1,) * rho.ndim) * rho[None] * (
        1.0 + eu / CS2 + (eu * eu - CS2 * uu[None]) / (CS2 * CS2))


def guo_force(Q, u, F):
    """Eq. e6: omega_i [(e_i - u)/cs2 + (u.e_i) e_i / cs4] . F."""
    e = velocities(Q).astype(np.float64)
    w = omega(Q)
    eu = np.tensordot(e, u, axes=(1, 0))
    eF = np.tensordot(e, F, axes=(1, 0))
    uF = (u * F).sum(axis=0)
    return w.reshape((Q,) + (1,) * (u.ndim - 1)) * ((eF - uF[None]) / CS2 + eu * eF / (CS2 * CS2))


def bgk_guo_collide(f, rho, u, F, tau, Q):
    """f* = f - (f - f^eq)/tau + (1 - 1/(2 tau)) F_bar, velocity space only."""
    feq = feq_hermite(Q, rho, u)
    Fb = guo_force(Q, u, F)
    return f - (f - feq) / tau + (1.0 - 0.5 / tau) * Fb


def lambda_collide(f, rho, u, F, forces, psi, p):
    """Eq. e7 with a dense Lambda = M^-1 S M (constant rates only)."""
    Q = p.lattice
    if p.variable_nu:
        raise ValueError("lambda_collide supports constant relaxation rates only")
    M, Minv = _mom.matrices(Q)
    S = np.diag(_mom.relaxation_vector(Q, p.rates))
    Lam = Minv @ S @ M
    feq = np.tensordot(Minv, _mom.equilibrium(Q, rho, u[0], u[1], u[2]), axes=(1, 0))
    Ft = _mom.forcing(Q, F[0], F[1], F[2], u[0], u[1], u[2])
    if p.eos != "none":
        t_nu = 1.0 / p.rates["s2"] - 0.5
        t_e = 1.0 / p.rates["s2b"] - 0.5
        Qxx, Qyy, Qzz, Qxy, Qxz, Qyz = forces["Q"]
        Fint2 = (forces["F_int"] ** 2).sum(axis=0)
        psi2 = psi * psi
        sig = np.where(psi2 > 0.0, 6.0 * p.sigma * Fint2 / np.where(psi2 > 0.0, psi2, 1.0) / t_e, 0.0)
        pos = lambda k: _mom.position(Q, k)  # noqa: E731
        Ft[pos(4)] -= Qxy / t_nu
        Ft[pos(5)] -= Qxz / t_nu
        Ft[pos(6)] -= Qyz / t_nu
        Ft[pos(7)] += sig + 4.0 * (Qxx + Qyy + Qzz) / (5.0 * t_e)
        Ft[pos(8)] -= (Qxx - Qyy) / t_nu
        Ft[pos(9)] -= (Qxx - Qzz) / t_nu
    Fb = np.tensordot(Minv, Ft, axes=(1, 0))
    I = np.eye(Q)
    return (f - np.tensordot(Lam, f - feq, axes=(1, 0))
            + np.tensordot(I - 0.5 * Lam, Fb, axes=(1, 0)))


def step_with(state, collide_fn):
    """Advance an ``lbm.State`` by one step using the given velocity-space collision."""
    rho, psi, forces, F, u = state.fields()
    fstar = collide_fn(state.f, rho, u, F, forces, psi)
    fstar = np.where(state.solid[None], 0.0, fstar)
    state.f = _lbm.stream(fstar, state.solid, state.p)
    state.t += 1
    return state
