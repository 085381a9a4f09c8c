"""One time step of the non-orthogonal MRT pseudopotential LBM (oracle; test infrastructure only).

All arrays are float64 numpy, shaped (nz, ny, nx) per field and (Q, nz, ny, nx)
for populations.  Velocity e_i = (e_x, e_y, e_z) shifts x by e_x etc.  The step
follows the paper's order:

1. rho = sum_i f_bar_i                                    (Sec. II A, after Eq. e9)
2. psi = sqrt(2 (p_EOS - rho c_s^2) / G)                  (Sec. II C)
3. F_int = -G psi(x) sum_i w_i psi(x + e_i) e_i           (Eq. e15)
   F_ads = -G_ads psi(x) sum_i w_i psi(x) s(x + e_i) e_i  (Sec. III E)
   Q_ab  = kappa G/2 psi(x) sum_i w_i [psi(x+e_i) - psi(x)] e_ia e_ib   (Eq. e18)
   F = F_int + F_ads + rho g                              (Eq. e6: F is the total force)
4. u = (sum_i f_bar_i e_i + F/2) / rho                    (Sec. II A)
5. m_bar = M f_bar; m^eq (Eq. e13); F~ (Eq. e14) modified by Eq. e17;
   m_bar* = m_bar - S (m_bar - m^eq) + (I - S/2) F~'      (Eq. e8)
6. f_bar* = M^-1 m_bar*                                   (Sec. II A)
7. f_bar_i(x + e_i, t + 1) = f_bar*_i(x, t)               (Eq. e9), half-way
   bounce-back where x + e_i is solid: f_bar_ibar(x, t+1) = f_bar*_i(x, t).

Readings where the paper is silent:
* s_e in Eq. e17 is the rate of m_7 (s2b); s_nu is the shear rate s2 (per cell when
  the viscosity varies with density, Sec. IV A).
* F_int in the sigma term of Eq. e17 is the interaction force alone.
* psi(x + e_i) at a solid neighbour is taken equal to psi(x) in Eq. e15 and Eq. e18,
  so that G_ads = 0 gives a neutral wall as Sec. III E states; wall effects then
  come only from F_ads.
* Walls on a non-periodic axis sit half-way outside the first and last planes.
* Solid cells carry no populations (zero) and report rho = 0, u = 0.
* The equation of state "none" means single-phase: no psi, F = rho g.

Parity: pinned (tests/test_oracle_lbm.py, tests/test_oracle_physics.py) by the
rest-state fixed point, mass and momentum conservation on periodic boxes,
independence of s0 and s1, equality with the independent velocity-space forms
of ``velocity_space`` (SRT BGK with Guo forcing, and Eq. e7 with a dense
Lambda), shear-wave decay at nu = (1/s2 - 1/2)/3, Poiseuille flow between
bounce-back walls, planar coexistence densities and interface width for the
piecewise EOS (Sec. III A), Laplace's law, the (1 - kappa) scaling of the
surface tension (Eq. ea18), and the neutral-wall fixed point.
"""
from dataclasses import dataclass, field

import numpy as np

from . import eos as _eos
from . import moments as _mom
from .lattice import CS2 as _CS2_EXACT
from .lattice import check_lattice, opposite, velocities, w_norm

CS2 = float(_CS2_EXACT)


@dataclass
class Params:
    lattice: int = 19
    shape: tuple = (16, 16, 16)            # (nx, ny, nz)
    bc: tuple = (0, 0, 0)                  # per axis x, y, z: 0 periodic, 1 walls at both ends
    eos: str = "none"                      # "none", "cs" or "piecewise"
    eos_p: tuple = ()                      # cs: (a, b, R, T); piecewise: (rho1, rho2, theta_v, theta_m, theta_l)
    G: float = -1.0                        # interaction strength (Sec. III A uses G = -1)
    G_ads: float = 0.0                     # fluid-solid strength (Sec. III E)
    kappa: float = 0.0                     # surface-tension tuning (Eq. e18)
    sigma: float = 0.0                     # mechanical-stability parameter (Eq. e17)
    rates: dict = field(default_factory=lambda: dict(_mom.DEFAULT_RATES))
    variable_nu: bool = False              # nu(rho) of Sec. IV A
    nu_l: float = 0.0
    nu_v: float = 0.0
    rho_l: float = 1.0
    rho_v: float = 0.0
    g: tuple = (0.0, 0.0, 0.0)             # body force per unit mass

    def validate(self):
        check_lattice(self.lattice)
        if self.eos not in ("none", "cs", "piecewise"):
            raise ValueError("eos must be none, cs or piecewise")
        if self.eos != "none" and self.G == 0.0:
            raise ValueError("a multiphase EOS needs G != 0")
        for k, v in self.rates.items():
            if not 0.0 < v < 2.0:
                raise ValueError(f"relaxation rate {k}={v} outside (0, 2)")


# ------------------------------------------------------------------ neighbour access
def _pad(field_, bc, fill):
    """field_ with one ghost layer on each of its last three axes (z, y, x): periodic wrap,
    or `fill` beyond a wall.  bc is given as (x, y, z)."""
    out = field_
    lead = field_.ndim - 3
    for axis, b in ((lead, bc[2]), (lead + 1, bc[1]), (lead + 2, bc[0])):
        widths = [(0, 0)] * out.ndim
        widths[axis] = (1, 1)
        if b == 0:
            out = np.pad(out, widths, mode="wrap")
        else:
            out = np.pad(out, widths, mode="constant", constant_values=fill)
    return out


def _at(padded, e, shape_zyx):
    """padded(x + e) for every interior x (e = (ex, ey, ez)), on the last three axes."""
    nz, ny, nx = shape_zyx
    ex, ey, ez = (int(c) for c in e)
    return padded[..., 1 + ez:1 + ez + nz, 1 + ey:1 + ey + ny, 1 + ex:1 + ex + nx]


# ------------------------------------------------------------------ step 1-2: density and psi
def density(f, solid):
    rho = f.sum(axis=0)
    return np.where(solid, 0.0, rho)


def pressure_eos(rho, p: Params):
    if p.eos == "cs":
        a, b, R, T = p.eos_p
        return _eos.cs_pressure(rho, a, b, R, T)
    if p.eos == "piecewise":
        return _eos.piecewise_pressure(rho, *p.eos_p)
    return rho * CS2


def pseudopotential(rho, solid, p: Params):
    """Square-root pseudopotential of Sec. II C on fluid cells (0 on solid cells and for eos 'none')."""
    if p.eos == "none":
        return np.zeros_like(rho)
    psi2 = _eos.psi_squared(pressure_eos(rho, p), rho, p.G)
    psi2 = np.where(solid, 0.0, psi2)
    if np.any(psi2 < 0.0):
        raise FloatingPointError("psi^2 < 0: density outside the range of the equation of state")
    return np.sqrt(psi2)


# ------------------------------------------------------------------ step 3: forces
def interaction(psi, solid, p: Params):
    """F_int (Eq. e15), F_ads (Sec. III E), Q_ab (Eq. e18) and S = sum_i w_i psi(x+e_i) e_i.

    Returns a dict of (3, ...) / (6, ...) arrays; Q components in the order xx, yy, zz, xy, xz, yz.
    """
    Q = p.lattice
    e = velocities(Q)
    w = w_norm(Q)
    shape = psi.shape
    if p.eos == "none":
        zero3 = np.zeros((3,) + shape)
        return dict(F_int=zero3, F_ads=zero3.copy(), Q=np.zeros((6,) + shape), S=zero3.copy())
    psi_pad = _pad(psi, p.bc, 0.0)
    sol_pad = _pad(solid, p.bc, True)
    S = np.zeros((3,) + shape)
    Sads = np.zeros((3,) + shape)
    Qab = np.zeros((6,) + shape)
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    for i in range(1, Q):
        s_nb = _at(sol_pad, e[i], shape)
        psi_nb = np.where(s_nb, psi, _at(psi_pad, e[i], shape))   # neutral continuation at solid neighbours
        for a in range(3):
            if e[i][a] != 0:
                S[a] += w[i] * psi_nb * e[i][a]
                Sads[a] += w[i] * s_nb * e[i][a]
        d = psi_nb - psi
        for c, (a, b) in enumerate(pairs):
            if e[i][a] != 0 and e[i][b] != 0:
                Qab[c] += w[i] * d * e[i][a] * e[i][b]
    F_int = -p.G * psi * S
    F_ads = -p.G_ads * psi * psi * Sads
    Qab = p.kappa * 0.5 * p.G * psi * Qab
    fluid = ~solid
    return dict(F_int=F_int * fluid, F_ads=F_ads * fluid, Q=Qab * fluid, S=S * fluid)


def total_force(rho, forces, p: Params):
    g = np.asarray(p.g, dtype=np.float64).reshape(3, 1, 1, 1)
    return forces["F_int"] + forces["F_ads"] + rho[None] * g


# ------------------------------------------------------------------ step 4: macroscopic
def velocity(f, rho, F, solid, Q):
    e = velocities(Q).astype(np.float64)
    j = np.tensordot(e.T, f, axes=(1, 0)) + 0.5 * F
    safe = np.where(solid, 1.0, rho)
    return np.where(solid[None], 0.0, j / safe[None])


def shear_rate(rho, p: Params):
    """s_nu = s2, or from nu(rho) = nu_v + (nu_l - nu_v)(rho - rho_v)/(rho_l - rho_v) (Sec. IV A)
    through nu = (1/s_nu - 1/2) c_s^2 (text after Eq. e12)."""
    if not p.variable_nu:
        return np.full(rho.shape, p.rates["s2"])
    nu = p.nu_v + (p.nu_l - p.nu_v) * (rho - p.rho_v) / (p.rho_l - p.rho_v)
    return 1.0 / (nu / CS2 + 0.5)


# ------------------------------------------------------------------ step 5-6: collision
def collide(f, rho, u, F, forces, psi, solid, p: Params):
    Q = p.lattice
    M, Minv = _mom.matrices(Q)
    m = np.tensordot(M, f, axes=(1, 0))
    meq = _mom.equilibrium(Q, rho, u[0], u[1], u[2])
    Ft = _mom.forcing(Q, F[0], F[1], F[2], u[0], u[1], u[2])

    s_nu = shear_rate(rho, p)
    s_e = p.rates["s2b"]
    if p.eos != "none":
        # Eq. e17, with (1/s - 0.5) dt for dt = 1
        t_nu = 1.0 / s_nu - 0.5
        t_e = 1.0 / s_e - 0.5
        Qxx, Qyy, Qzz, Qxy, Qxz, Qyz = forces["Q"]
        Fint2 = (forces["F_int"] ** 2).sum(axis=0)
        psi2 = psi * psi
        sig = np.where(psi2 > 0.0, 6.0 * p.sigma * Fint2 / np.where(psi2 > 0.0, psi2, 1.0) / t_e, 0.0)
        Ft[_mom.position(Q, 4)] -= Qxy / t_nu
        Ft[_mom.position(Q, 5)] -= Qxz / t_nu
        Ft[_mom.position(Q, 6)] -= Qyz / t_nu
        Ft[_mom.position(Q, 7)] += sig + 4.0 * (Qxx + Qyy + Qzz) / (5.0 * t_e)
        Ft[_mom.position(Q, 8)] -= (Qxx - Qyy) / t_nu
        Ft[_mom.position(Q, 9)] -= (Qxx - Qzz) / t_nu

    s = np.broadcast_to(_mom.relaxation_vector(Q, p.rates).reshape((Q,) + (1,) * rho.ndim),
                        (Q,) + rho.shape).copy()
    s[_mom.shear_mask(Q)] = s_nu
    mstar = m - s * (m - meq) + (1.0 - 0.5 * s) * Ft        # Eq. e8
    fstar = np.tensordot(Minv, mstar, axes=(1, 0))
    return np.where(solid[None], 0.0, fstar)


# ------------------------------------------------------------------ step 7: streaming
def stream(fstar, solid, p: Params):
    """Pull form of Eq. e9 with half-way bounce-back: the population arriving at x in
    direction i left x - e_i, unless x - e_i is solid, in which case it is the one x sent
    toward the solid in direction ibar, reflected."""
    Q = p.lattice
    e = velocities(Q)
    opp = opposite(Q)
    shape = solid.shape
    sol_pad = _pad(solid, p.bc, True)
    f_pad = _pad(fstar, p.bc, 0.0)
    out = np.empty_like(fstar)
    for i in range(Q):
        src = _at(f_pad[i], -e[i], shape)
        src_solid = _at(sol_pad, -e[i], shape)
        out[i] = np.where(src_solid, fstar[opp[i]], src)
    return np.where(solid[None], 0.0, out)


# ------------------------------------------------------------------ state
class State:
    """Populations f_bar (natural layout, post-streaming) plus the solid mask."""

    def __init__(self, params: Params, f, solid, t=0):
        params.validate()
        self.p = params
        self.f = f
        self.solid = solid
        self.t = t

    @classmethod
    def from_fields(cls, params: Params, rho, u, solid=None):
        """f_bar(t=0) = M^-1 m^eq(rho_0, u_0) (Eq. e13 through M^-1)."""
        params.validate()
        Q = params.lattice
        nx, ny, nz = params.shape
        rho = np.asarray(rho, dtype=np.float64).reshape(nz, ny, nx)
        u = np.asarray(u, dtype=np.float64).reshape(3, nz, ny, nx)
        solid = np.zeros((nz, ny, nx), dtype=bool) if solid is None else np.asarray(solid).astype(bool)
        _, Minv = _mom.matrices(Q)
        meq = _mom.equilibrium(Q, rho, u[0], u[1], u[2])
        f = np.tensordot(Minv, meq, axes=(1, 0))
        f = np.where(solid[None], 0.0, f)
        return cls(params, f, solid)

    def fields(self):
        """(rho, psi, forces, F, u) of the current populations."""
        rho = density(self.f, self.solid)
        psi = pseudopotential(rho, self.solid, self.p)
        forces = interaction(psi, self.solid, self.p)
        F = total_force(rho, forces, self.p)
        u = velocity(self.f, rho, F, self.solid, self.p.lattice)
        return rho, psi, forces, F, u

    def step(self):
        rho, psi, forces, F, u = self.fields()
        fstar = collide(self.f, rho, u, F, forces, psi, self.solid, self.p)
        self.f = stream(fstar, self.solid, self.p)
        self.t += 1

    def run(self, n):
        for _ in range(n):
            self.step()
        return self

    def moments(self):
        """(rho, u) with u = (sum f e + F/2)/rho at the current time (Sec. II A)."""
        rho, _, _, _, u = self.fields()
        return rho, u

    def sums(self):
        """Mass and momentum over fluid cells: (sum rho, sum rho u_x, sum rho u_y, sum rho u_z)."""
        rho, u = self.moments()
        return np.array([rho.sum(), (rho * u[0]).sum(), (rho * u[1]).sum(), (rho * u[2]).sum()])
