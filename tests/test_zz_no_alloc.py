"""lbm_field_totals_noalloc: the totals entry point for callers that must not allocate device
memory while they run (graph capture, pre-budgeted allocators, real-time loops).  It keeps its
scratch in a fixed device array instead of calling cudaMalloc.  Checked through the C ABI against
the FP64 totals that lbm_get_moments computes from the populations, on two calls in a row."""
import ctypes

import numpy as np
import pytest

import workloads as W
from tests import parity_util as U

pytestmark = pytest.mark.gpu


def test_totals_without_allocation_match_get_moments():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2306_16274_gb300 import lbm as L

    shape = (40, 36, 28)
    kw, rl, rv = U.cs_eos("T0.7")
    d = dict(lattice=19, shape=shape, sigma=0.1, kappa=0.3, g=(1e-5, -2e-5, 0.0), **kw)
    rho, u = W.droplet(shape, 8.0, rl, rv)
    sim = U.run_gpu(d, rho, u, steps=10)
    totals = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    seen = []
    for _ in range(2):
        sim.step(5)
        r, uu, sums = sim.moments()              # existing path: totals from the populations
        L.field_totals_noalloc(r, uu, totals)    # new path: totals of the rho / u fields
        torch.cuda.synchronize()
        got = totals.cpu().numpy()
        rd, ud = r.double().cpu().numpy(), uu.double().cpu().numpy()
        # the fields carry FP32 u = j / rho, so rho u differs from j by FP32 rounding per cell
        scale = np.array([rd.sum()] + [(rd * np.abs(ud[a])).sum() for a in range(3)])
        assert np.all(np.abs(got - sums) <= 1e-6 * scale + 1e-12), (got, sums)
        seen.append(got)
    assert not np.array_equal(seen[0], seen[1])   # the state moved between the two calls

    # sizes beyond the fixed scratch are rejected before any launch, with a message
    lib = L.lib()
    st = lib.lbm_field_totals_noalloc(r.data_ptr(), uu.data_ptr(), 33554433, totals.data_ptr(), None)
    assert st == 1 and b"33554432" in lib.lbm_last_error(None)
    st = lib.lbm_field_totals_noalloc(None, uu.data_ptr(), 10, totals.data_ptr(), None)
    assert st == 1
