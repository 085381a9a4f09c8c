"""Contact observables of droplet impact, FP64/numpy (TEST INFRASTRUCTURE ONLY).

Sec. III E measures the contact time of a droplet bouncing off a super-hydrophobic
wall and the spreading film radius; Sec. IV B the contact time on a wall carrying
a cylinder.  The paper defines both in words only, so this module writes out the
reading used throughout:

* a fluid cell is liquid when rho > threshold, the mid density (rho_l + rho_v) / 2;
* a fluid cell touches a solid when one of its lattice neighbours x + e_i (the active
  lattice's velocities, i != 0) is a solid cell of the mask or lies beyond a wall;
* contact: at least one liquid cell touches a solid; the contact time runs from the first
  step with contact to the first later step without contact that stays without contact for
  `hold` steps (a hydrophobic wall can hold a spreading film one cell above it on a vapour
  cushion for a while before the droplet leaves; hold = 0 takes the first step without);
* the footprint on a bottom wall is the set of liquid cells in the layer z = 0; the
  spreading diameter D_f is the mean of its x and y extents (cells).

``contact`` returns the same six numbers as the library's contact detector, so the two can
be compared cell count for cell count on the same density field (taken in float32 on both
sides, since the comparison decides an integer).  Pinned by brute force on small hand-made
fields in tests/test_oracle_observe.py.
"""
import numpy as np

from . import lattice
from .lbm import _at, _pad

INT32_MAX = 2 ** 31 - 1
INT32_MIN = -2 ** 31


def touches_solid(solid, bc, Q):
    """bool (nz, ny, nx): fluid cells with a solid lattice neighbour (mask or wall)."""
    solid = np.asarray(solid, dtype=bool)
    padded = _pad(solid, bc, True)
    e = lattice.velocities(Q)
    out = np.zeros(solid.shape, dtype=bool)
    for i in range(1, Q):
        out |= _at(padded, e[i], solid.shape)
    return out & ~solid


def contact(rho, solid, bc, Q, threshold):
    """[wet, floor, xmin, xmax, ymin, ymax] as ints (see module header); rho (nz, ny, nx)
    compared with threshold in rho's own precision."""
    rho = np.asarray(rho)
    nz, ny, nx = rho.shape
    solid = np.zeros(rho.shape, dtype=bool) if solid is None else np.asarray(solid, dtype=bool)
    thr = rho.dtype.type(threshold)
    wet = touches_solid(solid, bc, Q) & (rho > thr)
    out = [int(wet.sum()), 0, INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN]
    if bc[2] == 1:
        fl = wet[0]
        out[1] = int(fl.sum())
        if out[1]:
            ys, xs = np.nonzero(fl)
            out[2:] = [int(xs.min()), int(xs.max()), int(ys.min()), int(ys.max())]
    return out


def spreading_diameter(c):
    """D_f from a contact record: mean of the footprint's x and y extents (0 without one)."""
    if c[1] == 0:
        return 0.0
    return 0.5 * ((c[3] - c[2] + 1) + (c[5] - c[4] + 1))


def contact_time(wet_counts, steps, hold=0):
    """(touch, detach) steps from a series of wet-cell counts taken at `steps`: touch = first
    step with wet > 0; detach = the first later step with wet == 0 from which the counts stay
    0 for at least `hold` steps (None where not reached)."""
    touch = None
    zero_from = None
    for w, t in zip(wet_counts, steps):
        if touch is None:
            if w > 0:
                touch = t
            continue
        if w > 0:
            zero_from = None
            continue
        if zero_from is None:
            zero_from = t
        if t - zero_from >= hold:
            return touch, zero_from
    return touch, None
