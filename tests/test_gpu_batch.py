"""Multi-domain batches (lbm_batch_*): every member must evolve bitwise as when stepped alone,
whatever the grouping, tiling, graph replay or tuning."""
import numpy as np
import pytest

import workloads as W
from tests import parity_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _members():
    """(params dict, rho, u, solid) for a mixed set: both lattices, periodic droplets, a walled
    impact with interior solids, a single-phase domain, ragged sizes."""
    kw7, rl7, rv7 = U.cs_eos("T0.7")
    kwp, rlp, rvp = U.pw_eos()
    out = []
    shape = (37, 21, 18)
    out.append((dict(lattice=19, shape=shape, sigma=0.1, kappa=0.3, **kw7), *W.droplet(shape, 6.0, rl7, rv7), None))
    shape = (33, 30, 26)
    out.append((dict(lattice=27, shape=shape, sigma=0.1, **kw7), *W.droplet(shape, 7.0, rl7, rv7), None))
    shape = (40, 18, 22)
    rho, u = W.impact(shape, 6.0, rlp, rvp, U=0.03, gap=3.0)
    solid = W.cylinder_mask(shape, 3.0, axis="y")
    out.append((dict(lattice=19, shape=shape, bc=(0, 0, 1), sigma=0.1, G_ads=0.1, **kwp), rho, u, solid))
    shape = (24, 24, 30)
    rho, u = W.impact(shape, 5.0, rl7, rv7, U=0.02, gap=3.0)
    out.append((dict(lattice=27, shape=shape, bc=(0, 0, 1), sigma=0.1, G_ads=-0.05, **kw7), rho, u, None))
    shape = (29, 11, 13)
    out.append((dict(lattice=19, shape=shape, g=(1e-5, 0.0, 0.0)), *W.perturbed(shape, seed=4), None))
    shape = (48, 40, 36)
    out.append((dict(lattice=19, shape=shape, sigma=0.1, kappa=0.5, **kw7), *W.droplet(shape, 9.0, rl7, rv7), None))
    return out


def _make(members):
    return [U.run_gpu(d, rho, u, solid) for (d, rho, u, solid) in members]


@pytest.mark.parametrize("nsteps", [1, 2, 7, 40])
def test_batch_equals_members_stepped_alone(nsteps):
    from paper_2306_16274_gb300 import Batch
    m = _members()
    alone = _make(m)
    together = _make(m)
    for s in alone:
        s.step(nsteps)
    b = Batch(together)
    b.step(nsteps)
    b.sync()
    info = b.info()
    # groups: one per (lattice, solid handling, physics); a member with walls or solids has its
    # solid-free tiles in a plain group and the others in a solid group
    assert info["groups"] == 8
    if nsteps >= 2:
        assert info["graph_mode"] in (1, 2)
    for a, t in zip(alone, together):
        assert t.step_count == a.step_count == nsteps
        assert np.array_equal(a.populations().cpu().numpy(), t.populations().cpu().numpy())
        ra, ua, _ = a.moments()
        rt, ut, _ = t.moments()
        assert np.array_equal(ra.cpu().numpy(), rt.cpu().numpy())
    b.close()


def test_batch_replay_and_tuning_keep_results():
    # several graph launches (recorded once), a tuning pass that re-tiles every group, more steps
    from paper_2306_16274_gb300 import Batch
    m = _members()
    alone = _make(m)
    together = _make(m)
    b = Batch(together)
    b.step(6)
    b.step(5)
    choice = b.tune(trial_steps=2)
    assert len(choice) == b.info()["groups"]
    b.step(8)
    b.sync()
    total = together[0].step_count
    assert total == 6 + 5 + 12 * 3 + 8     # the tuner advances 12 x (trial_steps + 1) steps
    for a in alone:
        a.step(total)
    for a, t in zip(alone, together):
        assert np.array_equal(a.populations().cpu().numpy(), t.populations().cpu().numpy())
    b.close()


def test_batch_member_against_oracle():
    from paper_2306_16274_gb300 import Batch
    (d, rho, u, solid) = _members()[2]          # walled impact with a cylinder, piecewise EOS
    sim = U.run_gpu(d, rho, u, solid)
    b = Batch([sim])
    b.step(60)
    b.sync()
    ref = U.run_oracle(d, rho, u, solid, steps=60)
    er, eu, _, _ = U.compare_moments(sim, ref)
    assert er < 1e-4 and eu < 1e-4, (er, eu)
    b.close()


def test_batch_rejects_mixed_phases_and_duplicates():
    from paper_2306_16274_gb300 import Batch, LBMError
    m = _members()[:2]
    sims = _make(m)
    sims[0].step(1)
    with pytest.raises(LBMError) as e:
        Batch(sims)
    assert e.value.status == 7
    with pytest.raises(LBMError):
        Batch([sims[1], sims[1]])
    sims[1].step(1)
    b = Batch(sims)
    sims[0].step(1)                              # stepped apart after the batch was made
    with pytest.raises(LBMError) as e:
        b.step(2)
    assert e.value.status == 7
    b.close()


def test_batch_groups_share_physics_and_regroup_on_new_mask():
    # members with equal physics share one launch per pass, whatever their shapes; a member
    # re-initialised with a solid mask moves to a solid-handling group at the next step
    from paper_2306_16274_gb300 import Batch
    kw7, rl7, rv7 = U.cs_eos("T0.7")
    m = []
    for shape, r in (((37, 21, 18), 6.0), ((40, 33, 20), 7.0), ((16, 16, 16), 4.0)):
        m.append((dict(lattice=19, shape=shape, sigma=0.1, kappa=0.3, **kw7), *W.droplet(shape, r, rl7, rv7), None))
    alone = _make(m)
    together = _make(m)
    b = Batch(together)
    assert b.info()["groups"] == 1
    b.step(4)                                   # even: re-initialising restarts at AA phase 0
    for a in alone:
        a.step(4)
    d, _, _, _ = m[1]
    rho, u = W.droplet(d["shape"], 7.0, rl7, rv7)
    solid = W.cylinder_mask(d["shape"], 3.0, axis="z")
    import torch
    for s in (alone[1], together[1]):
        s.init_fields(torch.tensor(rho, dtype=torch.float32, device="cuda"),
                      torch.tensor(u, dtype=torch.float32, device="cuda"),
                      torch.tensor(solid, dtype=torch.uint8, device="cuda"))
    b.step(6)
    b.sync()
    assert b.info()["groups"] == 2
    for a in alone:
        a.step(6)
    for a, t in zip(alone, together):
        assert np.array_equal(a.populations().cpu().numpy(), t.populations().cpu().numpy())
    b.close()


@pytest.mark.parametrize("which", [2, 3])
def test_single_domain_tile_path_equals_grid_path(which):
    # a domain with walls or solids steps through its own one-member batch (solid-free tiles
    # without solid handling); with kernel timing on it takes the whole-grid kernels instead.
    # Both must give the same bits.
    d, rho, u, solid = _members()[which]
    tiles = U.run_gpu(d, rho, u, solid)
    grid = U.run_gpu(d, rho, u, solid)
    grid.set_kernel_timing(True)
    for n in (7, 40):
        tiles.step(n)
        grid.step(n)
        assert np.array_equal(tiles.populations().cpu().numpy(), grid.populations().cpu().numpy())
    ms, launches = grid.kernel_timing()
    assert launches["collide"] == 47 and launches["psi"] == 47


def test_groups_larger_than_one_launch():
    # 70 members of one physics with walls in z: the solid-free and the solid-handling group each hold
    # 70 members, more than one launch's member table (64), so each pass runs two launches per group,
    # with their own collide tiles, density tiles and density runs (widths 33 / 40 / 47 add narrow
    # columns).  Every member evolves bitwise as when stepped alone.
    from paper_2306_16274_gb300 import Batch
    kw, rl, rv = U.cs_eos("T0.7")
    members = []
    for k in range(70):
        shape = (33 + 7 * (k % 3), 9 + k % 4, 6 + k % 3)
        rho, u = W.droplet(shape, 2.5 + 0.5 * (k % 2), rl, rv)
        members.append((dict(lattice=19, shape=shape, bc=(0, 0, 1), sigma=0.1, kappa=0.3, G_ads=0.05, **kw), rho, u,
                        None))
    alone = _make(members)
    together = _make(members)
    b = Batch(together)
    assert b.info()["groups"] == 2
    for n in (1, 5):
        b.step(n)
        b.sync()
        for a in alone:
            a.step(n)
        for k, (a, t) in enumerate(zip(alone, together)):
            assert np.array_equal(a.populations().cpu().numpy(), t.populations().cpu().numpy()), (k, n)
    b.close()
    for sim in alone + together:
        sim.close()


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("nx", [33, 44, 48])
def test_narrow_columns_next_to_walls_and_solids(Q, nx):
    # nx = 32 + 1 .. 16: the last cells of every row step in 16-wide tiles; here they touch a wall in
    # x (walls on every face) and a solid cylinder crosses them.  The one-member batch (tiles,
    # solid handling only where needed) equals the whole-grid kernels (solid handling everywhere) bit
    # for bit, and both follow the oracle.
    kw, rl, rv = U.cs_eos("T0.7")
    shape = (nx, 14, 10)
    rho, u = W.droplet(shape, 4.0, rl, rv)
    z, y, x = np.meshgrid(np.arange(10), np.arange(14), np.arange(nx), indexing="ij")
    solid = ((x - (nx - 5)) ** 2 + (y - 7) ** 2 <= 2.5 ** 2).astype(np.uint8)   # a post along z near x = nx
    d = dict(lattice=Q, shape=shape, bc=(1, 1, 1), sigma=0.1, kappa=0.3, G_ads=0.05, **kw)
    tiles = U.run_gpu(d, rho, u, solid)
    grid = U.run_gpu(d, rho, u, solid)
    grid.set_kernel_timing(True)
    for n in (3, 20):
        tiles.step(n)
        grid.step(n)
        assert np.array_equal(tiles.populations().cpu().numpy(), grid.populations().cpu().numpy()), n
    ref = U.run_oracle(d, rho, u, solid, steps=23)
    er, eu, _, _ = U.compare_moments(tiles, ref)
    assert er < 1e-4 and eu < 1e-4, (er, eu)


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("shape,zchunk", [((40, 20, 3), 0), ((33, 17, 26), 0), ((33, 17, 26), 5)])
def test_zwall_domain_split_equals_batch(Q, shape, zchunk):
    # a domain with walls only at the z ends steps its inner planes with the solid-free kernel and
    # the two wall planes with the solid kernel; stepping it alone must equal stepping it as the
    # only member of a batch (tiles classified by solid need) bit for bit
    from paper_2306_16274_gb300 import Batch
    kw, rl, rv = U.cs_eos("T0.7")
    nx, ny, nz = shape
    rho, u = W.impact(shape, min(nx, ny, 2 * nz) / 5.0, rl, rv, U=0.05, gap=0.5)
    d = dict(lattice=Q, shape=shape, bc=(0, 0, 1), sigma=0.1, kappa=0.3, G_ads=0.1, zchunk=zchunk, **kw)
    a = U.run_gpu(d, rho, u, steps=0)
    b = U.run_gpu(d, rho, u, steps=0)
    bb = Batch([b])
    for n in (1, 4, 9):
        a.step(n)
        bb.step(n)
        assert np.array_equal(a.populations(device=False), b.populations(device=False)), (n,)


def test_every_tile_shape_equals_members_stepped_alone():
    # each compiled tile shape of the multi-domain kernels (32 x 4, 32 x 2, 16 x 8, 16 x 4, and 32 x 4
    # at fewer resident blocks) forced on every group, with automatic and fixed z-chunks: the members
    # still evolve bitwise as when stepped alone, after odd and even step counts
    from paper_2306_16274_gb300 import Batch
    from paper_2306_16274_gb300.lbm import lib
    nshapes = 5
    m = _members()
    alone = _make(m)
    for s in alone:
        s.step(3 * nshapes)
    together = _make(m)
    b = Batch(together)
    for shape in range(nshapes):
        for g in range(b.info()["groups"]):
            b.set_group(g, shape, 0 if shape % 2 == 0 else 3)
        assert all(gr["shape"] == shape for gr in b.groups())
        b.step(3)
    b.sync()
    for a, t in zip(alone, together):
        assert np.array_equal(a.populations().cpu().numpy(), t.populations().cpu().numpy())
    # unknown shapes and groups are refused
    with pytest.raises(Exception):
        b.set_group(0, nshapes, 0)
    with pytest.raises(Exception):
        b.set_group(b.info()["groups"], 0, 0)
    assert lib().lbm_batch_group(b._b, -1, None, None, None, None) == 1
    b.close()


def test_tuner_picks_a_shape_per_group_and_keeps_results():
    from paper_2306_16274_gb300 import Batch
    m = _members()
    alone = _make(m)
    together = _make(m)
    b = Batch(together)
    zc = b.tune(trial_steps=1)
    groups = b.groups()
    assert len(zc) == len(groups) == b.info()["groups"]
    assert all(0 <= g["shape"] < 5 and g["zchunk"] == z for g, z in zip(groups, zc))
    tuned_steps = together[0].step_count
    for s in alone:
        s.step(tuned_steps + 4)
    b.step(4)
    b.sync()
    for a, t in zip(alone, together):
        assert np.array_equal(a.populations().cpu().numpy(), t.populations().cpu().numpy())
    b.close()


def test_mixed_shapes_across_groups_keep_partners_aligned():
    # different shapes on different groups: a member's solid-free and solid groups are cut into the
    # same columns (setting one sets the other), so its cells are still covered exactly once
    from paper_2306_16274_gb300 import Batch
    m = _members()
    alone = _make(m)
    together = _make(m)
    b = Batch(together)
    n = b.info()["groups"]
    for g in range(n):
        b.set_group(g, (g * 2 + 1) % 5, g % 3)
    b.step(9)
    b.sync()
    for s in alone:
        s.step(9)
    for a, t in zip(alone, together):
        assert np.array_equal(a.populations().cpu().numpy(), t.populations().cpu().numpy())
    b.close()
