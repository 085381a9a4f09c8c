"""Moment-space algebra of the non-orthogonal MRT scheme (oracle; test infrastructure only).

* raw moments k_mnp = sum_i f_i e_ix^m e_iy^n e_iz^p          (Sec. II A, Eq. e2)
* the 27-element moment set m                                  (Sec. II B, Eq. e11)
* the transformation matrix M built from those definitions      (Eq. "matrix")
* its exact rational inverse by Gauss-Jordan elimination        (Sec. II B; the paper
  prints no M^-1, it sends the reader to supplementary material)
* the diagonal relaxation matrix S                              (Eq. e12)
* equilibrium moments m^eq                                      (Eq. e13)
* forcing moments F~                                            (Eq. e14)
* the D3Q19 model by extraction of rows/columns/elements        (App. C)

Pins (tests/test_oracle_moments.py): M equals the matrices printed in Sec. II B
and App. C (transcribed in tests/golden/); non-zero counts of M and M^-1 equal
Table I; M M^-1 = I in exact arithmetic; the D3Q19 M^-1 equals the restricted
D3Q27 M^-1 (App. C); m^eq = M f^eq with f^eq of Eq. e5 (D3Q27); F~ = M F_bar
with F_bar of Eq. e6 (D3Q27).
"""
from fractions import Fraction

import numpy as np

from .lattice import CS2, check_lattice, velocities

# Eq. e11: each moment is a signed sum of raw moments k_mnp, listed as (coef, (m, n, p)).
MOMENT_SET_27 = (
    ((1, (0, 0, 0)),),                                    # 0  k000 (density)
    ((1, (1, 0, 0)),),                                    # 1  k100
    ((1, (0, 1, 0)),),                                    # 2  k010
    ((1, (0, 0, 1)),),                                    # 3  k001
    ((1, (1, 1, 0)),),                                    # 4  k110
    ((1, (1, 0, 1)),),                                    # 5  k101
    ((1, (0, 1, 1)),),                                    # 6  k011
    ((1, (2, 0, 0)), (1, (0, 2, 0)), (1, (0, 0, 2))),     # 7  k200 + k020 + k002
    ((1, (2, 0, 0)), (-1, (0, 2, 0))),                    # 8  k200 - k020
    ((1, (2, 0, 0)), (-1, (0, 0, 2))),                    # 9  k200 - k002
    ((1, (1, 2, 0)),),                                    # 10 k120
    ((1, (1, 0, 2)),),                                    # 11 k102
    ((1, (2, 1, 0)),),                                    # 12 k210
    ((1, (2, 0, 1)),),                                    # 13 k201
    ((1, (0, 1, 2)),),                                    # 14 k012
    ((1, (0, 2, 1)),),                                    # 15 k021
    ((1, (1, 1, 1)),),                                    # 16 k111
    ((1, (2, 2, 0)),),                                    # 17 k220
    ((1, (2, 0, 2)),),                                    # 18 k202
    ((1, (0, 2, 2)),),                                    # 19 k022
    ((1, (2, 1, 1)),),                                    # 20 k211
    ((1, (1, 2, 1)),),                                    # 21 k121
    ((1, (1, 1, 2)),),                                    # 22 k112
    ((1, (1, 2, 2)),),                                    # 23 k122
    ((1, (2, 1, 2)),),                                    # 24 k212
    ((1, (2, 2, 1)),),                                    # 25 k221
    ((1, (2, 2, 2)),),                                    # 26 k222
)

# App. C: the D3Q19 moment set keeps moments 0..15 and k220, k202, k022 of Eq. e11.
D3Q19_MOMENTS = tuple(range(16)) + (17, 18, 19)


def moment_indices(Q):
    check_lattice(Q)
    return tuple(range(27)) if Q == 27 else D3Q19_MOMENTS


def matrix_exact(Q):
    """M as nested lists of ints: M[k][i] = sum over the raw moments of moment k of
    coef * e_ix^m e_iy^n e_iz^p (Eqs. e2, e11)."""
    e = velocities(Q)
    rows = []
    for k in moment_indices(Q):
        row = []
        for i in range(Q):
            ex, ey, ez = (int(c) for c in e[i])
            row.append(sum(c * ex ** m * ey ** n * ez ** p for c, (m, n, p) in MOMENT_SET_27[k]))
        rows.append(row)
    return rows


def inverse_exact(A):
    """Exact inverse of an integer/rational square matrix by Gauss-Jordan elimination
    with Fractions (no floating point anywhere)."""
    n = len(A)
    aug = [[Fraction(v) for v in row] + [Fraction(int(i == j)) for j in range(n)]
           for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if aug[r][col] != 0)
        aug[col], aug[piv] = aug[piv], aug[col]
        p = aug[col][col]
        aug[col] = [v / p for v in aug[col]]
        for r in range(n):
            if r != col and aug[r][col] != 0:
                fac = aug[r][col]
                aug[r] = [a - fac * b for a, b in zip(aug[r], aug[col])]
    return [row[n:] for row in aug]


_CACHE = {}


def matrices(Q):
    """(M, M^-1) as float64 arrays.  M^-1 is the exact rational inverse rounded once."""
    if Q not in _CACHE:
        Mx = matrix_exact(Q)
        Mi = inverse_exact(Mx)
        _CACHE[Q] = (np.array(Mx, dtype=np.float64),
                     np.array([[float(v) for v in row] for row in Mi], dtype=np.float64),
                     Mx, Mi)
    M, Minv, _, _ = _CACHE[Q]
    return M, Minv


def matrices_exact(Q):
    matrices(Q)
    return _CACHE[Q][2], _CACHE[Q][3]


RATE_NAMES = ("s0", "s1", "s2", "s2b", "s3", "s3b", "s4", "s4b", "s5", "s6")
# Defaults stated after Eq. e12: s0 = s1 = 1, s2b = s3b = 0.6, all others 1.2.
DEFAULT_RATES = dict(s0=1.0, s1=1.0, s2=1.2, s2b=0.6, s3=1.2, s3b=0.6, s4=1.2, s4b=1.2, s5=1.2, s6=1.2)

# Eq. e12: which rate relaxes each of the 27 moments.
RATE_OF_MOMENT_27 = ("s0", "s1", "s1", "s1", "s2", "s2", "s2", "s2b", "s2", "s2",
                     "s3", "s3", "s3", "s3", "s3", "s3", "s3b", "s4", "s4", "s4",
                     "s4b", "s4b", "s4b", "s5", "s5", "s5", "s6")
# moments relaxed with the shear rate s_nu = s2 (used for variable viscosity and Eq. e17)
SHEAR_MOMENTS_27 = (4, 5, 6, 8, 9)


def relaxation_vector(Q, rates):
    """diag(S) of Eq. e12 (D3Q19: App. C, the same rates restricted)."""
    return np.array([rates[RATE_OF_MOMENT_27[k]] for k in moment_indices(Q)], dtype=np.float64)


def shear_mask(Q):
    """Boolean vector over the Q moments: True where the rate is s_nu (= s2)."""
    idx = moment_indices(Q)
    return np.array([k in SHEAR_MOMENTS_27 for k in idx])


def equilibrium_27(rho, ux, uy, uz):
    """m^eq of Eq. e13 (27 entries), element-wise over arrays."""
    cs2 = float(CS2)
    cs4, cs6 = cs2 * cs2, cs2 * cs2 * cs2
    u2 = ux * ux + uy * uy + uz * uz
    z = np.zeros_like(rho)
    return np.stack([
        rho, rho * ux, rho * uy, rho * uz,
        rho * ux * uy, rho * ux * uz, rho * uy * uz,
        rho * (1.0 + u2), rho * (ux * ux - uy * uy), rho * (ux * ux - uz * uz),
        rho * cs2 * ux, rho * cs2 * ux, rho * cs2 * uy, rho * cs2 * uz, rho * cs2 * uy, rho * cs2 * uz,
        z,
        rho * cs2 * (cs2 + ux * ux + uy * uy), rho * cs2 * (cs2 + ux * ux + uz * uz),
        rho * cs2 * (cs2 + uy * uy + uz * uz),
        rho * cs2 * uy * uz, rho * cs2 * ux * uz, rho * cs2 * ux * uy,
        rho * cs4 * ux, rho * cs4 * uy, rho * cs4 * uz,
        rho * cs4 * u2 + rho * cs6,
    ])


def forcing_27(Fx, Fy, Fz, ux, uy, uz):
    """F~ of Eq. e14 (27 entries), element-wise over arrays."""
    cs2 = float(CS2)
    cs4 = cs2 * cs2
    Fu = Fx * ux + Fy * uy + Fz * uz
    z = np.zeros_like(Fx * ux)
    return np.stack([
        z, Fx + z, Fy + z, Fz + z,
        Fx * uy + Fy * ux, Fx * uz + Fz * ux, Fy * uz + Fz * uy,
        2.0 * Fu, 2.0 * (Fx * ux - Fy * uy), 2.0 * (Fx * ux - Fz * uz),
        Fx * cs2 + z, Fx * cs2 + z, Fy * cs2 + z, Fz * cs2 + z, Fy * cs2 + z, Fz * cs2 + z,
        z,
        2.0 * cs2 * (Fx * ux + Fy * uy), 2.0 * cs2 * (Fx * ux + Fz * uz), 2.0 * cs2 * (Fy * uy + Fz * uz),
        cs2 * (Fy * uz + Fz * uy), cs2 * (Fx * uz + Fz * ux), cs2 * (Fx * uy + Fy * ux),
        cs4 * Fx + z, cs4 * Fy + z, cs4 * Fz + z,
        2.0 * cs4 * Fu,
    ])


def equilibrium(Q, rho, ux, uy, uz):
    """m^eq for the lattice: Eq. e13 for D3Q27; its extracted elements for D3Q19 (App. C)."""
    return equilibrium_27(rho, ux, uy, uz)[list(moment_indices(Q))]


def forcing(Q, Fx, Fy, Fz, ux, uy, uz):
    """F~ for the lattice: Eq. e14 for D3Q27; its extracted elements for D3Q19 (App. C)."""
    return forcing_27(Fx, Fy, Fz, ux, uy, uz)[list(moment_indices(Q))]


def position(Q, k27):
    """Position of moment k27 (index in Eq. e11) in the lattice's moment vector."""
    return moment_indices(Q).index(k27)
