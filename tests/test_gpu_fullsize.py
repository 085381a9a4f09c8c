"""Full-size checks in the launch configuration bench.py times: the 256^3 at-scale workload with
automatic z-chunks (each collide block marches through 26 planes on D3Q19, 20 on D3Q27).  Sampled cells are compared
with the oracle, which advances a small periodic sub-box around each sample: after one step a
cell depends only on the initial state within two cells (psi stencil of its pull sources), after
two steps within four, so a sub-box of radius 3 / 5 closed by walls reproduces the full-domain
result at its centre.  Conservation is checked over the whole domain."""
import numpy as np
import pytest

import bench
from oracle import lbm as olbm
from tests import parity_util as U

pytestmark = pytest.mark.gpu

SHAPE = (256, 256, 256)


@pytest.fixture(scope="module")
def workload():
    import __graft_entry__
    __graft_entry__.build()
    rho, u, wparams = bench.workload_fields(SHAPE)
    return rho, u, wparams


def _samples(rho, seed, n_interface=8, n_other=4):
    rng = np.random.default_rng(seed)
    lo, hi = rho.min(), rho.max()
    frac = (rho - lo) / (hi - lo)
    iface = np.argwhere((frac > 0.1) & (frac < 0.9))
    pick = iface[rng.choice(len(iface), n_interface, replace=False)]
    other = rng.integers(0, 256, size=(n_other, 3))
    edges = np.array([[0, 0, 0], [255, 255, 255], [0, 128, 255], [255, 7, 0]])   # periodic wrap in z, y, x
    return np.concatenate([pick, other, edges])


def _oracle_subbox(d, rho, u, center, radius, steps):
    # the sub-box is closed by bounce-back walls (a periodic wrap of a sub-box would join
    # mismatched densities); wall effects travel at most two cells per step, so the centre is
    # exact for radius >= 2 steps + 1
    z, y, x = (int(c) for c in center)
    idx = [np.arange(c - radius, c + radius + 1) % 256 for c in (z, y, x)]
    r = rho[np.ix_(*idx)]
    uu = u[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
    n = 2 * radius + 1
    dd = dict(d)
    dd["shape"] = (n, n, n)
    dd["bc"] = (1, 1, 1)
    s = U.run_oracle(dd, r, uu, steps=steps)
    return s.f[:, radius, radius, radius]


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("steps", [1, 2])
def test_sampled_cells_match_oracle(workload, Q, steps):
    import torch
    rho, u, wparams = workload
    d = dict(lattice=Q, shape=SHAPE, **wparams)
    sim = U.run_gpu(d, rho, u, steps=steps)
    f = sim.populations()
    samples = _samples(rho, seed=Q * 10 + steps)
    idx = torch.tensor(samples, device=f.device, dtype=torch.long)
    fg = f[:, idx[:, 0], idx[:, 1], idx[:, 2]].double().cpu().numpy()
    del f
    sim.close()
    torch.cuda.empty_cache()
    radius = 3 if steps == 1 else 5
    for k, c in enumerate(samples):
        fo = _oracle_subbox(d, rho, u, c, radius, steps)
        err = np.abs(fg[:, k] - fo).max()
        assert err < 2e-6 * np.abs(fo).max(), (tuple(c), err)


@pytest.mark.parametrize("Q", [19, 27])
def test_fullsize_conservation(workload, Q):
    # total mass (and total momentum, F_int being pairwise antisymmetric) is invariant on the
    # periodic box; FP32 populations drift only by rounding
    rho, u, wparams = workload
    d = dict(lattice=Q, shape=SHAPE, **wparams)
    sim = U.run_gpu(d, rho, u, steps=0)
    _, _, s0 = sim.moments()
    sim.step(200)
    sim.sync()
    _, _, s1 = sim.moments()
    sim.close()
    assert abs(s1[0] - s0[0]) < 1e-5 * s0[0]
    assert np.abs(s1[1:] - s0[1:]).max() < 1e-5 * s0[0]


@pytest.mark.parametrize("Q", [19, 27])
def test_fullsize_onepass_equals_two_pass(workload, Q):
    # the one-pass step in its bench configuration reproduces the two-pass step bit for bit over
    # both AA parities (compared on the device)
    import torch
    rho, u, wparams = workload
    d = dict(lattice=Q, shape=SHAPE, **wparams)
    a = U.run_gpu(d, rho, u, steps=3)
    fa = a.populations()
    a.close()
    b = U.run_gpu(dict(d, onepass=True), rho, u, steps=3)
    fb = b.populations()
    b.close()
    assert torch.equal(fa, fb)
    del fa, fb
    torch.cuda.empty_cache()


@pytest.mark.parametrize("Q", [19, 27])
def test_fullsize_fp16_paired_layout(workload, Q):
    # the shifted-FP16 store as the bench runs it (x-paired layout, pair kernels) against the one-cell
    # layout bit for bit after three steps, and sampled cells against the oracle at the FP16 bound
    import torch
    rho, u, wparams = workload
    d = dict(lattice=Q, shape=SHAPE, store="fp16", **wparams)
    a = U.run_gpu(d, rho, u, steps=3)
    fa = a.populations()
    a.close()
    b = U.run_gpu(dict(d, store_layout="single"), rho, u, steps=3)
    fb = b.populations()
    b.close()
    assert torch.equal(fa, fb)
    samples = _samples(rho, seed=Q * 100 + 3)
    idx = torch.tensor(samples, device=fa.device, dtype=torch.long)
    fg = fa[:, idx[:, 0], idx[:, 1], idx[:, 2]].double().cpu().numpy()
    del fa, fb
    torch.cuda.empty_cache()
    d32 = dict(lattice=Q, shape=SHAPE, **wparams)
    for k, c in enumerate(samples[:8]):
        fo = _oracle_subbox(d32, rho, u, c, 7, 3)
        assert np.abs(fg[:, k] - fo).max() < 1e-3 * np.abs(fo).max(), tuple(c)


def test_fullsize_batch_equals_jobs_stepped_alone():
    # the batched workload in the configuration bench.py times (64 jobs, 105.7 M cells, edges 48-160,
    # both lattices, periodic droplets and impacts on a wall), tuned and stepped as one batch: every
    # job's populations equal those of the job stepped alone, bit for bit (compared on the device)
    import torch

    from paper_2306_16274_gb300 import Batch, Params, Simulation
    jobs = bench.batch_jobs(64)

    def make():
        out = []
        for params, rho, u in jobs:
            s = Simulation(Params(**params))
            s.init_fields(torch.tensor(rho, dtype=torch.float32, device="cuda"),
                          torch.tensor(u, dtype=torch.float32, device="cuda"))
            out.append(s)
        return out

    together = make()
    b = Batch(together)
    b.tune(trial_steps=1)
    b.step(5)
    b.sync()
    b.close()
    total = together[0].step_count
    assert total == 12 * 2 + 5
    for k, t in enumerate(together):
        fb = t.populations()
        t.close()
        a = Simulation(Params(**jobs[k][0]))
        a.init_fields(torch.tensor(jobs[k][1], dtype=torch.float32, device="cuda"),
                      torch.tensor(jobs[k][2], dtype=torch.float32, device="cuda"))
        a.step(total)
        assert torch.equal(a.populations(), fb), k
        a.close()
        del fb
    torch.cuda.empty_cache()


def test_largest_domain_near_the_cell_limit():
    # 1290^3 = 2,146,689,000 cells, just under the 2^31 - 1 cells that 32-bit cell offsets allow
    # (D3Q19 populations 163 GB): two steps of a C-S field, sampled cells (among them the last
    # cell and the far corners) against the oracle on wall-closed sub-boxes, and mass conservation
    import torch
    n = 1290
    free, _ = torch.cuda.mem_get_info()
    if free < 215e9:
        pytest.skip(f"needs ~210 GB of free device memory, {free / 1e9:.0f} GB free")
    kw, rl, rv = U.cs_eos("T0.7")
    d = dict(lattice=19, shape=(n, n, n), sigma=0.1, kappa=0.3, **kw)
    gen = torch.Generator(device="cuda").manual_seed(2306)
    rho = 0.2 + 0.02 * torch.rand((n, n, n), device="cuda", generator=gen)
    u = 0.01 * (torch.rand((3, n, n, n), device="cuda", generator=gen) - 0.5)
    samples = np.array([[n - 1, n - 1, n - 1], [0, 0, 0], [n - 1, 0, n - 1], [0, n - 1, 0],
                        [n // 2, 7, n - 3], [1111, 1289, 3]])
    radius, steps = 5, 2
    windows = []
    for c in samples:
        idx = [torch.tensor([(int(v) + k) % n for k in range(-radius, radius + 1)], device="cuda") for v in c]
        r = rho.index_select(0, idx[0]).index_select(1, idx[1]).index_select(2, idx[2])
        uu = u.index_select(1, idx[0]).index_select(2, idx[1]).index_select(3, idx[2])
        windows.append((r.double().cpu().numpy(), uu.double().cpu().numpy()))
    from paper_2306_16274_gb300 import Simulation
    sim = Simulation(U.gpu_params(d))
    sim.init_fields(rho, u)
    del rho, u
    torch.cuda.empty_cache()
    _, _, s0 = sim.moments(device=True)
    torch.cuda.empty_cache()
    sim.step(steps)
    r_g, u_g, s1 = sim.moments(device=True)
    t = torch.tensor(samples, device="cuda", dtype=torch.long)
    rg = r_g[t[:, 0], t[:, 1], t[:, 2]].double().cpu().numpy()
    ug = u_g[:, t[:, 0], t[:, 1], t[:, 2]].double().cpu().numpy()
    del r_g, u_g
    sim.close()
    torch.cuda.empty_cache()
    m = 2 * radius + 1
    for k, (r, uu) in enumerate(windows):
        dd = dict(d)
        dd["shape"] = (m, m, m)
        dd["bc"] = (1, 1, 1)
        ro, uo = U.run_oracle(dd, r, uu, steps=steps).moments()
        assert abs(rg[k] - ro[radius, radius, radius]) < 2e-6 * ro[radius, radius, radius], (tuple(samples[k]),)
        assert np.abs(ug[:, k] - uo[:, radius, radius, radius]).max() < 2e-6, (tuple(samples[k]),)
    assert abs(s1[0] - s0[0]) < 1e-6 * s0[0]


@pytest.mark.parametrize("shape", [(65535, 3, 2), (2, 5, 65535)])
def test_maximum_extent(shape):
    # an axis at LBM_MAX_EXTENT (the psi pass launches one block row per z plane): two steps of a
    # C-S field, cells at both ends of the long axis against the oracle on wall-closed sub-boxes
    import torch
    nx, ny, nz = shape
    kw, rl, rv = U.cs_eos("T0.7")
    d = dict(lattice=27, shape=shape, sigma=0.1, **kw)
    rng = np.random.default_rng(65535)
    rho = 0.2 + 0.02 * rng.random((nz, ny, nx))
    u = 0.01 * (rng.random((3, nz, ny, nx)) - 0.5)
    radius, steps = 5, 2
    sim = U.run_gpu(d, rho, u, steps=steps)
    r_g, u_g, _ = sim.moments(device=False)
    sim.close()
    long_axis = int(np.argmax(shape))
    n_long = shape[long_axis]
    for pos in (0, 1, n_long // 2, n_long - 2, n_long - 1):
        c = [0, 0, 0]                     # (x, y, z)
        c[long_axis] = pos
        x, y, z = c
        idx = [np.arange(v - radius, v + radius + 1) % size for v, size in ((z, nz), (y, ny), (x, nx))]
        r = rho[np.ix_(*idx)]
        uu = u[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
        m = 2 * radius + 1
        dd = dict(d, shape=(m, m, m), bc=(1, 1, 1))
        ro, uo = U.run_oracle(dd, r, uu, steps=steps).moments()
        assert abs(r_g[z, y, x] - ro[radius, radius, radius]) < 2e-6 * ro[radius, radius, radius], (c,)
        assert np.abs(u_g[:, z, y, x] - uo[:, radius, radius, radius]).max() < 2e-6, (c,)


def test_allocation_failure_is_reported():
    # a context larger than the device (two D3Q27 population copies of 1290^3 cells, ~470 GB):
    # lbm_create frees what it allocated and returns LBM_ERR_OOM; the device stays usable
    import torch
    from paper_2306_16274_gb300 import LBMError, Simulation
    _, total = torch.cuda.mem_get_info()
    p = U.gpu_params(dict(lattice=27, shape=(1290, 1290, 1290), onepass=True))
    from paper_2306_16274_gb300 import estimate_bytes
    if estimate_bytes(p) <= total:
        pytest.skip("the device is large enough for this context")
    free0, _ = torch.cuda.mem_get_info()
    with pytest.raises(LBMError) as e:
        Simulation(p)
    assert e.value.status == 2
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20)
    sim = U.run_gpu(dict(lattice=19, shape=(8, 8, 8)), np.ones((8, 8, 8)), np.zeros((3, 8, 8, 8)), steps=2)
    sim.sync()
