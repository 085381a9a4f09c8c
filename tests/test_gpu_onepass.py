"""One-pass stepping over two population copies (lbm_params.onepass): the same arithmetic as the
in-place two-pass step (collide-stream, then density/psi), reordered so that each block computes
the density and psi it needs from the copy being read.  Every population, psi and moment must
equal the two-pass path's bit for bit, on ragged tiles, tiles wider than the domain and several
z-chunks; the two-pass path itself is checked against the FP64 oracle in the parity tests, and one
case here is checked against the oracle directly."""
import numpy as np
import pytest

import workloads as W
from tests import parity_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def cases():
    kw7, rl7, rv7 = U.cs_eos("T0.7")
    kwp, rlp, rvp = U.pw_eos()
    out = []
    shape = (24, 20, 16)
    out.append(("shear19", dict(lattice=19, shape=shape, rates={"s2": 1.1}), *W.shear_wave(shape, 0.05)))
    out.append(("tg27_narrow", dict(lattice=27, shape=(13, 7, 6)), *W.taylor_green((13, 7, 6), 0.04)))
    shape = (33, 30, 28)
    out.append(("drop19_cs", dict(lattice=19, shape=shape, sigma=0.1, kappa=0.3, **kw7),
                *W.droplet(shape, 8.0, rl7, rv7, W=3.0)))
    out.append(("drop27_cs_zc3", dict(lattice=27, shape=shape, sigma=0.1, zchunk=3, **kw7),
                *W.droplet(shape, 7.0, rl7, rv7, W=3.0)))
    shape = (40, 9, 21)
    out.append(("drop19_pw_g_varnu", dict(lattice=19, shape=shape, sigma=0.1, g=(0.0, 0.0, -1e-5),
                                          variable_nu=True, nu_l=0.1, nu_v=0.05, rho_l=rlp, rho_v=rvp, **kwp),
                *W.droplet(shape, 4.0, rlp, rvp, W=3.0)))
    shape = (18, 18, 5)
    out.append(("drop27_small_zc1", dict(lattice=27, shape=shape, sigma=0.05, zchunk=1, **kw7),
                *W.droplet(shape, 4.0, rl7, rv7, W=3.0)))
    return out


@pytest.mark.parametrize("case", cases(), ids=lambda c: c[0])
def test_onepass_is_bitwise_equal_to_two_pass(case):
    name, d, rho, u = case
    a = U.run_gpu(d, rho, u, steps=0)
    b = U.run_gpu(dict(d, onepass=True), rho, u, steps=0)
    for n in (1, 6, 37):
        a.step(n)
        b.step(n)
        assert a.step_count == b.step_count
        fa, fb = a.populations(device=False), b.populations(device=False)
        assert np.array_equal(fa, fb), (name, n, float(np.abs(fa - fb).max()))
        assert np.array_equal(a.psi(device=False), b.psi(device=False)), (name, n)
        ra, ua, sa = a.moments(device=False)
        rb, ub, sb = b.moments(device=False)
        assert np.array_equal(ra, rb) and np.array_equal(ua, ub) and list(sa) == list(sb)


def test_onepass_against_oracle():
    name, d, rho, u = cases()[2]
    sim = U.run_gpu(dict(d, onepass=True), rho, u, steps=100)
    ref = U.run_oracle(d, rho, u, steps=100)
    er, eu, sg, so = U.compare_moments(sim, ref)
    assert er < 1e-4 and eu < 1e-4, (er, eu)     # the multiphase parity bound of the two-pass path
    assert abs(sg[0] - so[0]) < 1e-6 * so[0]


def test_onepass_checkpoint_round_trip():
    import torch

    name, d, rho, u = cases()[3]
    a = U.run_gpu(dict(d, onepass=True), rho, u, steps=9)
    f = a.populations(device=True).clone()
    # restore into a one-pass and a two-pass context: both continue exactly as the original
    b = U.run_gpu(dict(d, onepass=True), rho, u, steps=0)
    c = U.run_gpu(d, rho, u, steps=0)
    b.set_populations(f)
    c.set_populations(f.cpu().numpy())
    assert torch.equal(b.populations(device=True), f)
    for s in (a, b, c):
        s.step(11)
    fa = a.populations(device=False)
    assert np.array_equal(fa, b.populations(device=False))
    assert np.array_equal(fa, c.populations(device=False))


def test_onepass_launch_count_and_single_pass_timing():
    name, d, rho, u = cases()[2]
    sim = U.run_gpu(dict(d, onepass=True), rho, u, steps=2)
    sim.set_kernel_timing(True)
    sim.step(5)
    ms, n = sim.kernel_timing()
    assert n == {"psi": 0, "collide": 5}
    assert ms["collide"] > 0


def test_onepass_rejects_solids_and_batches():
    import torch

    from paper_2306_16274_gb300 import Batch, LBMError
    name, d, rho, u = cases()[0]
    sim = U.run_gpu(dict(d, onepass=True), rho, u, steps=0)
    solid = torch.zeros(tuple(reversed(d["shape"])), dtype=torch.uint8, device="cuda")
    with pytest.raises(LBMError):
        sim.init_fields(torch.tensor(rho, dtype=torch.float32, device="cuda"),
                        torch.tensor(u, dtype=torch.float32, device="cuda"), solid)
    other = U.run_gpu(dict(d, onepass=True), rho, u, steps=0)
    with pytest.raises(LBMError):
        Batch([other])


def test_onepass_status_words():
    # the one pass evaluates the EOS itself: a density beyond the C-S range and a NaN density are
    # reported through the same status words as in the two-pass step
    from paper_2306_16274_gb300 import LBMError
    kw, rl, rv = U.cs_eos("T0.7")
    d = dict(lattice=19, shape=(8, 8, 8), sigma=0.1, onepass=True, **kw)
    with pytest.raises(LBMError) as e:
        U.run_gpu(d, np.full((8, 8, 8), 0.75), np.zeros((3, 8, 8, 8)), steps=1).sync()
    assert e.value.status == 5
    rho = np.full((8, 8, 8), 0.2)
    rho[3, 3, 3] = np.nan
    sim = U.run_gpu(dict(lattice=27, shape=(8, 8, 8), onepass=True), rho, np.zeros((3, 8, 8, 8)), steps=2)
    with pytest.raises(LBMError) as e:
        sim.sync()
    assert e.value.status == 4


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 16), (1, 5, 1), (2, 3, 1), (33, 1, 2)])
def test_onepass_degenerate_extents(Q, shape):
    # extents of 1 and 2 cells: a tile's border wraps onto the tile itself
    kw, rl, rv = U.cs_eos("T0.7")
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz)
    rho = 0.2 + 0.02 * rng.random((nz, ny, nx))
    u = 0.01 * (rng.random((3, nz, ny, nx)) - 0.5)
    d = dict(lattice=Q, shape=shape, sigma=0.1, kappa=0.3, **kw)
    a = U.run_gpu(d, rho, u, steps=5)
    b = U.run_gpu(dict(d, onepass=True), rho, u, steps=5)
    assert np.array_equal(a.populations(device=False), b.populations(device=False))


def _staged_cases():
    kw7, rl7, rv7 = U.cs_eos("T0.7")
    out = []
    shape = (64, 12, 9)        # two tiles in x (both at a face), three in y, z-chunks of 3 planes
    out.append(("drop19_64x12", dict(lattice=19, shape=shape, sigma=0.1, kappa=0.3, zchunk=3, g=(1e-5, 0.0, 0.0),
                                     **kw7), *W.droplet(shape, 4.0, rl7, rv7, W=3.0)))
    shape = (96, 16, 7)        # a tile away from the x faces
    out.append(("drop27_96x16", dict(lattice=27, shape=shape, sigma=0.1, zchunk=4, **kw7),
                *W.droplet(shape, 5.0, rl7, rv7, W=3.0)))
    shape = (32, 4, 5)         # one tile: all four faces at once
    out.append(("single19_32x4", dict(lattice=19, shape=shape, rates={"s2": 1.3}), *W.perturbed(shape, seed=5)))
    shape = (32, 8, 1)         # one plane: every staged plane is the same storage plane
    out.append(("single27_nz1", dict(lattice=27, shape=shape, g=(0.0, 2e-5, 0.0)), *W.perturbed(shape, seed=6)))
    return out


@pytest.mark.parametrize("case", _staged_cases(), ids=lambda c: c[0])
def test_staged_onepass_is_bitwise_equal_to_two_pass(case):
    # onepass = "staged" (nx a multiple of 32, ny of 4): the one-pass step stages each plane's pulled
    # populations with tensor copies (TMA) and fills the periodic images at the faces; results equal
    # the two-pass step
    name, d, rho, u = case
    a = U.run_gpu(d, rho, u, steps=0)
    b = U.run_gpu(dict(d, onepass="staged"), rho, u, steps=0)
    assert b.staged
    for n in (1, 6, 21):
        a.step(n)
        b.step(n)
        fa, fb = a.populations(device=False), b.populations(device=False)
        assert np.array_equal(fa, fb), (name, n, float(np.abs(fa - fb).max()))
        ra, ua, sa = a.moments(device=False)
        rb, ub, sb = b.moments(device=False)
        assert np.array_equal(ra, rb) and np.array_equal(ua, ub) and list(sa) == list(sb)


def test_staged_copy_waits_are_bounded():
    # a staged step that expects more bytes than its copies deliver: every wait runs out (about
    # 10 ms), the blocks abandon the step and LBM_ERR_TIMEOUT is reported; the context stays usable
    from paper_2306_16274_gb300 import LBMError
    name, d, rho, u = _staged_cases()[0]
    sim = U.run_gpu(dict(d, onepass="staged"), rho, u, steps=2)
    sim.debug_stage_timeout(True)
    sim.step(1)
    with pytest.raises(LBMError) as e:
        sim.sync()
    assert e.value.status == 6
    sim.debug_stage_timeout(False)
    ref = U.run_gpu(d, rho, u, steps=3)
    sim.init_fields(rho.astype(np.float32), u.astype(np.float32))
    sim.step(3)
    sim.sync()
    assert np.array_equal(sim.populations(device=False), ref.populations(device=False))
    # contexts that do not stage refuse the switch
    plain = U.run_gpu(dict(lattice=19, shape=(64, 8, 4), onepass=True), *W.perturbed((64, 8, 4), seed=1))
    assert not plain.staged
    with pytest.raises(LBMError):
        plain.debug_stage_timeout(True)
