"""Shifted FP16 population store (lbm_params.store = LBM_STORE_FP16): every result against the
FP64 oracle at tolerances derived from the storage precision, checkpoint round trip, memory
estimate, contact detection, and the batch restriction.

The tolerances: a slot keeps h = f / rho_w - omega in half precision (relative step 2^-11 of
|h| <= ~0.1, so about 5e-5 of f per write); 100 steps of independent roundings with the
collision's damping give the 1e-4-scale errors that an FP16 emulation of the oracle shows on
the same cases (liquid and vapour density within 2e-4, velocity within 6e-4 of its scale).
The bounds below leave a factor of about 5 above that."""
import numpy as np
import pytest

import workloads as W
from tests import parity_util as U

pytestmark = pytest.mark.gpu

TOL_RHO = 1e-3    # max over cells of |rho_fp16 - rho_oracle| / rho_oracle (vapour included)
TOL_U = 3e-3      # max |u_fp16 - u_oracle| / velocity scale


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def errors(sim, ref):
    r_g, u_g, sums = sim.moments(device=False)
    r_o, u_o = ref.moments()
    fluid = r_o > 0
    er = float((np.abs(r_g.astype(np.float64) - r_o)[fluid] / r_o[fluid]).max())
    scale = max(float(np.abs(u_o).max()), getattr(ref, "u0max", 0.0))
    eu = float(np.abs(u_g.astype(np.float64) - u_o).max() / scale)
    return er, eu, sums, ref.sums()


def cases():
    kw7, rl7, rv7 = U.cs_eos("T0.7")
    kwp, rlp, rvp = U.pw_eos()
    out = []
    shape = (24, 20, 16)
    out.append(("shear19", dict(lattice=19, shape=shape, rates={"s2": 1.1}), *W.shear_wave(shape, 0.05), None))
    out.append(("tg27", dict(lattice=27, shape=(20, 20, 6)), *W.taylor_green((20, 20, 6), 0.04), None))
    shape = (32, 30, 28)
    out.append(("drop19_cs", dict(lattice=19, shape=shape, sigma=0.1, kappa=0.3, **kw7),
                *W.droplet(shape, 8.0, rl7, rv7, W=3.0), None))
    out.append(("drop27_cs", dict(lattice=27, shape=shape, sigma=0.1, **kw7), *W.droplet(shape, 7.0, rl7, rv7, W=3.0),
                None))
    shape = (40, 36, 24)
    rho, u = W.impact(shape, 7.0, rlp, rvp, U=0.05, gap=2.0)
    out.append(("impact19_pw", dict(lattice=19, shape=shape, bc=(0, 0, 1), sigma=0.1, **kwp), rho, u, None))
    shape = (36, 32, 30)
    rho, u, solid = W.cylinder_impact(shape, 6.0, 5.0, rl7, rv7, 0.05, gap=2.0, W=3.0)
    out.append(("cyl27_cs", dict(lattice=27, shape=shape, bc=(0, 0, 1), sigma=0.1, kappa=0.3, G_ads=0.1, **kw7),
                rho, u, solid))
    return out


@pytest.mark.parametrize("case", cases(), ids=lambda c: c[0])
def test_fp16_store_against_oracle(case):
    name, d, rho, u, solid = case
    steps = 100
    d16 = dict(d, store="fp16", zchunk=3)
    sim = U.run_gpu(d16, rho, u, solid, steps=steps)
    ref = U.run_oracle(d, rho, u, solid, steps=steps)
    er, eu, sg, so = errors(sim, ref)
    mass = abs(sg[0] - so[0]) / so[0]
    print(f"\nFP16 {name} after {steps} steps: rho rel {er:.2e}, u rel {eu:.2e}, mass rel {mass:.2e}")
    assert er < TOL_RHO and eu < TOL_U, (er, eu)
    assert mass < 1e-4


def test_fp16_checkpoint_round_trip_and_estimate():
    import torch

    from paper_2306_16274_gb300 import estimate_bytes
    name, d, rho, u, solid = cases()[5]
    d16 = dict(d, store="fp16")
    sim = U.run_gpu(d16, rho, u, solid, steps=15)
    assert sim.device_bytes == estimate_bytes(U.gpu_params(d16), with_solid=True)
    f = sim.populations()
    other = U.run_gpu(d16, rho, u, solid)
    other.set_populations(f)
    g = other.populations()
    # re-storing rounds each value once more relative to the current densities
    scale = torch.clamp(f.abs(), min=1e-3 * float(f.abs().max()))
    assert float(((g - f).abs() / scale).max()) < 2e-3
    sim.step(20)
    other.step(20)
    ra, _, _ = sim.moments(device=False)
    rb, _, _ = other.moments(device=False)
    fl = ra > 0
    assert float((np.abs(ra - rb)[fl] / ra[fl]).max()) < 1e-3


def test_fp16_contact_matches_oracle_definition():
    from oracle import observe
    name, d, rho, u, solid = cases()[5]
    sim = U.run_gpu(dict(d, store="fp16"), rho, u, solid, steps=60)
    r, _, _ = sim.moments(device=False)
    thr = 0.5 * (U.cs_eos("T0.7")[1] + U.cs_eos("T0.7")[2])
    got = sim.contact(thr)
    assert list(got.values()) == observe.contact(r, solid, (0, 0, 1), 27, thr)


def test_fp16_contexts_cannot_join_a_batch():
    from paper_2306_16274_gb300 import Batch, LBMError
    name, d, rho, u, solid = cases()[2]
    sim = U.run_gpu(dict(d, store="fp16"), rho, u, solid)
    with pytest.raises(LBMError) as e:
        Batch([sim])
    assert e.value.status == 1


def _paired_cases():
    kw, rl, rv = U.cs_eos("T0.7")
    kwp, rlp, rvp = U.pw_eos()
    out = []
    for Q in (19, 27):
        # hx = 17: one ragged tile of pairs; hx = 35: a full and a ragged tile; z-chunks of 3 planes
        for shape in ((34, 11, 9), (70, 6, 7)):
            rho, u = W.droplet(shape, 3.0, rl, rv, W=3.0)
            out.append((f"drop{Q}_{shape[0]}", dict(lattice=Q, shape=shape, sigma=0.1, kappa=0.3, zchunk=3,
                                                    g=(1e-5, 0.0, 0.0), **kw), rho, u))
        shape = (40, 12, 10)
        rho, u = W.impact(shape, 4.0, rlp, rvp, U=0.05, gap=2.0)
        out.append((f"zwall{Q}", dict(lattice=Q, shape=shape, bc=(0, 1, 1), sigma=0.1, G_ads=0.1, zchunk=3, **kwp),
                    rho, u))
        # nx = 2: one word per row, both halves exchanged by every x shift
        r = 0.2 + 0.02 * np.random.default_rng(3).random((3, 5, 2))
        out.append((f"nx2_{Q}", dict(lattice=Q, shape=(2, 5, 3), sigma=0.1, **kw), r, np.zeros((3, 3, 5, 2))))
    return out


@pytest.mark.parametrize("case", _paired_cases(), ids=lambda c: c[0])
def test_fp16_paired_layout_equals_single_cell_kernels(case):
    # even nx, x periodic, no mask: the FP16 slots live two cells per word and step with the pair
    # kernels; store_layout "single" keeps one slot per cell and the one-cell kernels on the same
    # domain.  Both must give the same populations, psi and moments bit for bit, after odd and
    # even step counts.
    name, d, rho, u = case
    d16 = dict(d, store="fp16")
    paired = U.run_gpu(d16, rho, u)
    single = U.run_gpu(dict(d16, store_layout="single"), rho, u)
    for n in (1, 1, 5):
        paired.step(n)
        single.step(n)
        assert np.array_equal(paired.populations(device=False), single.populations(device=False)), (name, n)
        assert np.array_equal(paired.psi(device=False), single.psi(device=False)), (name, n)
        ra, ua, sa = paired.moments(device=False)
        rb, ub, sb = single.moments(device=False)
        assert np.array_equal(ra, rb) and np.array_equal(ua, ub) and np.array_equal(sa, sb), (name, n)
    # a checkpoint restores into either layout
    f = paired.populations(device=False)
    single.set_populations(f)
    paired.set_populations(f)
    paired.step(3)
    single.step(3)
    assert np.array_equal(paired.populations(device=False), single.populations(device=False)), name
