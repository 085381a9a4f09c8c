"""Runs a set of small cases through whichever liblbm.so LBM_LIBRARY names and prints one JSON line:
a digest of every case's final populations and the library's count of out-of-bounds accesses
(lbm_debug_bounds_violations; nonzero only in a bounds-checked build).  Used by
tests/test_gpu_bounds.py to compare a bounds-checked build with the normal one."""
import hashlib
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as W  # noqa: E402
from tests import parity_util as U  # noqa: E402


def digest(sim):
    return hashlib.sha256(np.ascontiguousarray(sim.populations(device=False)).tobytes()).hexdigest()[:16]


def main():
    from paper_2306_16274_gb300 import Batch, lib
    kw, rl, rv = U.cs_eos("T0.7")
    kwp, rlp, rvp = U.pw_eos()
    out = {}
    for Q in (19, 27):
        shape = (33, 30, 28)
        rho, u = W.droplet(shape, 8.0, rl, rv, W=3.0)
        d = dict(lattice=Q, shape=shape, sigma=0.1, kappa=0.3, zchunk=5, **kw)
        out[f"periodic{Q}"] = digest(U.run_gpu(d, rho, u, steps=7))
        out[f"onepass{Q}"] = digest(U.run_gpu(dict(d, onepass=True), rho, u, steps=7))
        # the one-pass step with tensor-copy staging and face images (nx a multiple of 32, ny of 4)
        ss = (64, 12, 9)
        rs, us = W.droplet(ss, 4.0, rl, rv, W=3.0)
        out[f"onepass_staged{Q}"] = digest(U.run_gpu(dict(d, shape=ss, onepass="staged"), rs, us, steps=7))
        out[f"fp16_{Q}"] = digest(U.run_gpu(dict(d, store="fp16"), rho, u, steps=7))
        # even nx: the x-paired FP16 layout and its pair kernels, periodic and with y / z walls
        sp = (34, 30, 28)
        rp, up = W.droplet(sp, 8.0, rl, rv, W=3.0)
        out[f"fp16p_{Q}"] = digest(U.run_gpu(dict(d, shape=sp, store="fp16"), rp, up, steps=7))
        out[f"fp16pw_{Q}"] = digest(U.run_gpu(dict(d, shape=sp, store="fp16", bc=(0, 1, 1)), rp, up, steps=7))
        shape = (40, 36, 24)
        rho, u = W.impact(shape, 7.0, rlp, rvp, U=0.05, gap=2.0)
        dw = dict(lattice=Q, shape=shape, bc=(0, 0, 1), sigma=0.1, G_ads=0.1, **kwp)
        out[f"zwalls{Q}"] = digest(U.run_gpu(dw, rho, u, steps=7))
        shape = (36, 32, 30)
        rho, u, solid = W.cylinder_impact(shape, 6.0, 5.0, rl, rv, 0.05, gap=2.0, W=3.0)
        dc = dict(lattice=Q, shape=shape, bc=(0, 0, 1), sigma=0.1, kappa=0.3, G_ads=0.1, **kw)
        out[f"cylinder{Q}"] = digest(U.run_gpu(dc, rho, u, solid, steps=7))
        a = U.run_gpu(dict(d, shape=(21, 13, 9)), *W.droplet((21, 13, 9), 3.0, rl, rv, W=3.0))
        b = U.run_gpu(dw, *W.impact((40, 36, 24), 7.0, rlp, rvp, U=0.05, gap=2.0))
        bb = Batch([a, b])
        bb.step(5)
        bb.sync()
        out[f"batch{Q}"] = digest(a) + digest(b)
        for shape in ((1, 1, 1), (2, 5, 3)):
            nx, ny, nz = shape
            r = 0.2 + 0.02 * np.random.default_rng(7).random((nz, ny, nx))
            v = np.zeros((3, nz, ny, nx))
            out[f"tiny{Q}_{nx}{ny}{nz}"] = digest(U.run_gpu(dict(lattice=Q, shape=shape, sigma=0.1, **kw), r, v, steps=3))
    shape = (65535, 3, 2)
    r = 0.2 + 0.02 * np.random.default_rng(65535).random((2, 3, 65535))
    out["extent"] = digest(U.run_gpu(dict(lattice=19, shape=shape, sigma=0.1, **kw), r, np.zeros((3, 2, 3, 65535)),
                                     steps=2))
    print(json.dumps({"digests": out, "violations": int(lib().lbm_debug_bounds_violations())}))


if __name__ == "__main__":
    main()
