"""Discrete velocity sets and weights (oracle; test infrastructure only).

D3Q27 velocities in the fixed order of Sec. II A, Eq. e1; D3Q19 is the first 19
of them (App. C).  Weights omega(|e|^2) for D3Q27 are given in the text after
Eq. e5.  The paper prints no D3Q19 weights; the standard D3Q19 set
(1/3, 1/18, 1/36) is used, which only enters through the normalised weights
w = omega / c_s^2 of Eq. e15 / Eq. e18 (a reading; the same isotropy
sum_i w e_ia e_ib = delta_ab holds for both lattices).

Pinned by tests/test_oracle_lattice.py: velocity order against the printed
matrix M (first three moment rows equal e_x, e_y, e_z), isotropy of the weights,
sum of weights equal to one.
"""
from fractions import Fraction

import numpy as np

# Eq. e1: |e_ix>, |e_iy>, |e_iz> for i = 0..26
EX27 = (0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1)
EY27 = (0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1)
EZ27 = (0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1)

CS2 = Fraction(1, 3)  # lattice sound speed squared, c_s = 1/sqrt(3) (Sec. II A)

# omega(|e|^2) for D3Q27 (text after Eq. e5)
OMEGA27 = {0: Fraction(8, 27), 1: Fraction(2, 27), 2: Fraction(1, 54), 3: Fraction(1, 216)}
# standard D3Q19 weights (not printed in the paper; see module docstring)
OMEGA19 = {0: Fraction(1, 3), 1: Fraction(1, 18), 2: Fraction(1, 36)}


def check_lattice(Q):
    if Q not in (19, 27):
        raise ValueError(f"lattice must be 19 or 27, got {Q}")


def velocities(Q):
    """(Q, 3) int array of (e_x, e_y, e_z); D3Q19 = first 19 of D3Q27 (App. C)."""
    check_lattice(Q)
    return np.array([EX27[:Q], EY27[:Q], EZ27[:Q]], dtype=np.int64).T.copy()


def opposite(Q):
    """Index of -e_i for every i."""
    e = velocities(Q)
    opp = []
    for i in range(Q):
        j = [k for k in range(Q) if tuple(e[k]) == tuple(-e[i])]
        assert len(j) == 1
        opp.append(j[0])
    return np.array(opp, dtype=np.int64)


def omega_exact(Q):
    """Weights omega_i as Fractions."""
    check_lattice(Q)
    table = OMEGA27 if Q == 27 else OMEGA19
    e = velocities(Q)
    return [table[int((e[i] ** 2).sum())] for i in range(Q)]


def omega(Q):
    return np.array([float(w) for w in omega_exact(Q)])


def w_norm(Q):
    """Normalised weights w(|e_i|^2) = omega(|e_i|^2) / c_s^2 of Eq. e15."""
    return np.array([float(w / CS2) for w in omega_exact(Q)])
