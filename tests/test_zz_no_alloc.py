"""lbm_field_totals_noalloc: the totals entry point for callers that cannot allocate device memory
while they run (a host whose device memory is handed out up front by its own pool allocator, a
real-time loop that may not block on cudaMalloc / cudaFree).  It keeps its scratch in a fixed device
array instead of calling cudaMalloc.  Checked through the C ABI, on two calls in a row, against the
FP64 totals that the existing entry point lbm_get_moments computes from the populations, and against
an FP64 host sum of the very rho / u arrays it was given.  The cell count is ragged (not a multiple of
the 2048 cells one block sums), so the last block is partly empty."""
import ctypes

import numpy as np
import pytest

import workloads as W
from tests import parity_util as U

pytestmark = pytest.mark.gpu


def _host_totals(rd, ud):
    """FP64 sums of the given float32 fields, exactly rounded per term (math.fsum)."""
    import math
    r = rd.reshape(-1).astype(np.float64)
    uu = ud.reshape(3, -1).astype(np.float64)
    return np.array([math.fsum(r)] + [math.fsum(r * uu[a]) for a in range(3)])


def test_totals_without_allocation_match_get_moments():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2306_16274_gb300 import lbm as L

    shape = (41, 37, 29)                      # 43,993 cells: 21 full blocks and a partial one
    assert (41 * 37 * 29) % 2048 != 0
    kw, rl, rv = U.cs_eos("T0.7")
    d = dict(lattice=19, shape=shape, sigma=0.1, kappa=0.3, g=(1e-5, -2e-5, 3e-6), **kw)
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
        rd, ud = r.cpu().numpy(), uu.cpu().numpy()
        # the same arrays summed on the host in FP64: only the order of the FP64 additions differs
        host = _host_totals(rd, ud)
        scale = np.array([np.abs(rd.astype(np.float64)).sum()] +
                         [(np.abs(rd.astype(np.float64)) * np.abs(ud[a].astype(np.float64))).sum() for a in range(3)])
        assert np.all(np.abs(got - host) <= 1e-12 * scale), (got, host)
        # against lbm_get_moments: its momentum is sum (sum f e + F/2) per cell, while the fields
        # carry the FP32 u = j / rho, so rho u differs from j by FP32 rounding per cell
        assert np.all(np.abs(got - sums) <= 1e-6 * scale + 1e-12), (got, sums)
        seen.append(got)
    assert not np.array_equal(seen[0], seen[1])   # the state moved between the two calls

    lib = L.lib()
    # sizes beyond the fixed scratch are rejected before any launch, with a message
    st = lib.lbm_field_totals_noalloc(r.data_ptr(), uu.data_ptr(), 33554433, totals.data_ptr(), None)
    assert st == 1 and b"33554432" in lib.lbm_last_error(None)
    st = lib.lbm_field_totals_noalloc(r.data_ptr(), uu.data_ptr(), 0, totals.data_ptr(), None)
    assert st == 1
    st = lib.lbm_field_totals_noalloc(None, uu.data_ptr(), 10, totals.data_ptr(), None)
    assert st == 1
    # a host array in place of a device one is refused before any launch
    host_rho = np.zeros(16, dtype=np.float32)
    st = lib.lbm_field_totals_noalloc(host_rho.ctypes.data, uu.data_ptr(), 16, totals.data_ptr(), None)
    assert st == 1 and b"current device" in lib.lbm_last_error(None)
    # the binding refuses what the C side could not check (dtype, contiguity) and CPU tensors
    with pytest.raises(ValueError):
        L.field_totals_noalloc(r.double(), uu, totals)
    with pytest.raises(ValueError):
        L.field_totals_noalloc(r, uu, totals.float())
    with pytest.raises(ValueError):
        L.field_totals_noalloc(r.cpu(), uu, totals)
    with pytest.raises(ValueError):
        L.field_totals_noalloc(r, uu.transpose(1, 2), totals)
    # a refused call leaves the last result in place
    torch.cuda.synchronize()
    assert np.array_equal(totals.cpu().numpy(), seen[1])
