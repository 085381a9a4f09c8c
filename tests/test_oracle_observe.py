"""Pins of the oracle's contact observables (Sec. III E / Sec. IV B, read in oracle/observe.py):
brute force over cells and lattice links, hand-counted cases, and the lattice dependence."""
import itertools

import numpy as np
import pytest

from oracle import observe

# e_i of D3Q27 written out independently of the oracle's tables: D3Q19 = |e|^2 <= 2
E27 = [e for e in itertools.product((-1, 0, 1), repeat=3) if e != (0, 0, 0)]
E19 = [e for e in E27 if sum(c * c for c in e) <= 2]


def brute_contact(rho, solid, bc, Q, thr):
    nz, ny, nx = rho.shape
    dirs = E19 if Q == 19 else E27
    wet = 0
    floor = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if solid[z, y, x] or not rho[z, y, x] > thr:
                    continue
                touch = False
                for ex, ey, ez in dirs:
                    p = [x + ex, y + ey, z + ez]
                    beyond = False
                    for a, n in enumerate((nx, ny, nz)):
                        if p[a] < 0 or p[a] >= n:
                            if bc[a] == 1:
                                beyond = True
                            p[a] %= n
                    if beyond or solid[p[2], p[1], p[0]]:
                        touch = True
                        break
                if touch:
                    wet += 1
                    if bc[2] == 1 and z == 0:
                        floor.append((x, y))
    out = [wet, len(floor), 2 ** 31 - 1, -2 ** 31, 2 ** 31 - 1, -2 ** 31]
    if floor:
        xs, ys = zip(*floor)
        out[2:] = [min(xs), max(xs), min(ys), max(ys)]
    return out


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("bc", [(0, 0, 1), (1, 0, 0), (0, 0, 0), (1, 1, 1)])
def test_contact_matches_brute_force(Q, bc):
    rng = np.random.default_rng(7 + Q + 3 * sum(bc))
    shape = (5, 6, 7)                      # (nz, ny, nx)
    rho = rng.uniform(0.0, 1.0, shape).astype(np.float32)
    solid = rng.uniform(size=shape) < 0.08
    got = observe.contact(rho, solid, bc, Q, 0.5)
    assert got == brute_contact(rho, solid, bc, Q, np.float32(0.5))


def test_contact_hand_counted_floor_patch():
    # 5 x 5 x 3 cells, walls in z: a 3 x 2 liquid patch on the floor touches the bottom wall;
    # a liquid cell in the middle plane touches nothing
    rho = np.zeros((3, 5, 5), dtype=np.float32)
    rho[0, 1:3, 1:4] = 1.0
    rho[1, 4, 4] = 1.0
    out = observe.contact(rho, None, (0, 0, 1), 19, 0.5)
    assert out == [6, 6, 1, 3, 1, 2]
    assert observe.spreading_diameter(out) == pytest.approx(0.5 * (3 + 2))


def test_contact_lattice_dependence():
    # a cell whose only solid neighbour is across a cube corner touches it on D3Q27 only
    rho = np.ones((4, 4, 4), dtype=np.float32)
    solid = np.zeros((4, 4, 4), dtype=bool)
    solid[0, 0, 0] = True
    rho[:] = 0.0
    rho[1, 1, 1] = 1.0
    assert observe.contact(rho, solid, (0, 0, 0), 19, 0.5)[0] == 0
    assert observe.contact(rho, solid, (0, 0, 0), 27, 0.5)[0] == 1
    rho[1, 1, 1] = 0.0
    rho[1, 1, 0] = 1.0                      # an edge neighbour: both lattices
    assert observe.contact(rho, solid, (0, 0, 0), 19, 0.5)[0] == 1
    assert observe.contact(rho, solid, (0, 0, 0), 27, 0.5)[0] == 1


def test_contact_threshold_is_strict_and_solid_cells_never_count():
    rho = np.full((3, 3, 3), 0.5, dtype=np.float32)
    solid = np.zeros((3, 3, 3), dtype=bool)
    solid[1, 1, 1] = True
    assert observe.contact(rho, solid, (0, 0, 0), 27, 0.5)[0] == 0
    rho[:] = 0.75
    assert observe.contact(rho, solid, (0, 0, 0), 27, 0.5)[0] == 26
    assert observe.contact(rho, solid, (0, 0, 0), 19, 0.5)[0] == 18


def test_contact_time_sequence():
    steps = [0, 10, 20, 30, 40, 50]
    assert observe.contact_time([0, 0, 4, 9, 0, 3], steps) == (20, 40)
    assert observe.contact_time([0, 1, 2, 3, 4, 5], steps) == (10, None)
    assert observe.contact_time([0] * 6, steps) == (None, None)
    # a lift-off shorter than the hold is not a detachment; the final one is, from its start
    steps = list(range(0, 120, 10))
    wet = [0, 5, 7, 0, 0, 6, 4, 0, 0, 0, 0, 0]
    assert observe.contact_time(wet, steps, hold=0) == (10, 30)
    assert observe.contact_time(wet, steps, hold=20) == (10, 70)
    assert observe.contact_time(wet, steps, hold=40) == (10, 70)
    assert observe.contact_time(wet, steps, hold=50) == (10, None)
