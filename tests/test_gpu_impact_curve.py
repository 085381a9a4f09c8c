"""Spreading diameter of a droplet hitting a flat wall (the down-scaled impact case of Sec. III E /
IV A): the GPU with FP32 populations and with the shifted-FP16 store against the FP64 oracle's
curve in tests/golden/impact_curve.json (written by tests/golden/make_impact_curve.py, which
calls only the oracle).  D_f is the mean of two integer extents, so it moves in half cells: each
sample may differ by at most one cell and the curves by at most 1 % on average."""
import json
import os

import numpy as np
import pytest

import workloads as W
from tests import parity_util as U
from tests.golden import make_impact_curve as G

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "impact_curve.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("store", ["fp32", "fp16"])
def test_spreading_diameter_against_oracle(store):
    ref = json.load(open(GOLDEN))
    kwp, rl, rv = U.pw_eos()
    d = dict(lattice=19, shape=G.SHAPE, bc=(0, 0, 1), sigma=0.1, kappa=0.0, store=store,
             rates={"s2": 1.0 / (3.0 * G.NU + 0.5), "s4": 1.0}, **kwp)
    rho, u = G.fields()
    sim = U.run_gpu(d, rho, u)
    thr = 0.5 * (rl + rv)
    df = []
    for _ in ref["steps"]:
        sim.step(G.EVERY)
        c = sim.contact(thr)
        df.append(0.0 if c["floor"] == 0 else 0.5 * ((c["xmax"] - c["xmin"] + 1) + (c["ymax"] - c["ymin"] + 1)))
    df, want = np.array(df), np.array(ref["D_f"])
    print(f"\n{store}: D_f/R0 {np.round(df / G.R0, 3).tolist()}\n oracle {np.round(want / G.R0, 3).tolist()}")
    assert np.abs(df - want).max() <= 1.0
    assert float(np.mean(np.abs(df - want) / np.maximum(want, 1.0))) <= 0.01
