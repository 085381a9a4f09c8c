"""Pins for oracle/lattice.py: velocity order and weights (Sec. II A, Eq. e1; App. C)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import lattice as la


def _printed(golden_dir, name):
    rows = [r for r in open(os.path.join(golden_dir, name)) if not r.startswith("#")]
    return np.array([[int(v) for v in r.split()] for r in rows])


@pytest.mark.parametrize("Q,name", [(27, "M27_printed.txt"), (19, "M19_printed.txt")])
def test_velocity_order_matches_printed_momentum_rows(golden_dir, Q, name):
    # rows 1..3 of the printed M are k100, k010, k001, i.e. e_x, e_y, e_z in the paper's order
    M = _printed(golden_dir, name)
    e = la.velocities(Q)
    assert (M[1] == e[:, 0]).all() and (M[2] == e[:, 1]).all() and (M[3] == e[:, 2]).all()
    assert len({tuple(v) for v in e}) == Q


@pytest.mark.parametrize("Q", [19, 27])
def test_weights_normalised_and_isotropic(Q):
    w = la.omega_exact(Q)
    e = la.velocities(Q)
    assert sum(w) == 1
    cs2 = la.CS2
    for a in range(3):
        for b in range(3):
            s2 = sum(w[i] * int(e[i][a]) * int(e[i][b]) for i in range(Q))
            assert s2 == (cs2 if a == b else 0)
    # fourth-order isotropy: sum w e_a^4 = 3 cs^4, sum w e_a^2 e_b^2 = cs^4
    for a in range(3):
        assert sum(w[i] * int(e[i][a]) ** 4 for i in range(Q)) == 3 * cs2 * cs2
        for b in range(a + 1, 3):
            assert sum(w[i] * int(e[i][a]) ** 2 * int(e[i][b]) ** 2 for i in range(Q)) == cs2 * cs2
    # normalised weights of Eq. e15: sum w e e = identity
    wn = la.w_norm(Q)
    ee = np.einsum("i,ia,ib->ab", wn, e, e)
    assert np.allclose(ee, np.eye(3), atol=1e-15)


def test_d3q27_weights_as_printed():
    # text after Eq. e5: omega(0)=8/27, omega(1)=2/27, omega(2)=1/54, omega(3)=1/216
    w = la.omega_exact(27)
    e = la.velocities(27)
    for i in range(27):
        n = int((e[i] ** 2).sum())
        assert w[i] == {0: Fraction(8, 27), 1: Fraction(2, 27), 2: Fraction(1, 54), 3: Fraction(1, 216)}[n]


@pytest.mark.parametrize("Q", [19, 27])
def test_opposite_is_involution(Q):
    opp = la.opposite(Q)
    e = la.velocities(Q)
    assert (opp[opp] == np.arange(Q)).all()
    assert (e[opp] == -e).all()
    with pytest.raises(ValueError):
        la.velocities(15)
