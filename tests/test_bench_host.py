"""Host-side pieces of bench.py: the algorithmic bytes per cell update the roofline divides by
(counted here from the populations each pass reads and writes), the whole-job rate, the committed
traffic record's source check, and the reference arm's oracle timing over several processes."""
import json
import os

import pytest

import bench


@pytest.mark.parametrize("Q", [19, 27])
def test_algorithmic_bytes(Q):
    pop = 4 * Q                                  # one FP32 population set
    b = bench.algorithmic_bytes(Q)
    assert b["collide"] == 2 * pop + 4           # read and write the populations, read psi
    assert b["psi"] == pop + 4                   # read the populations, write psi
    assert b["step"] == b["collide"] + b["psi"]
    h = bench.algorithmic_bytes(Q, "fp16")
    assert h["collide"] == 2 * (2 * Q) + 3 * 4   # 2-byte slots; densities read twice, psi once
    assert h["psi"] == 2 * Q + 3 * 4             # slots, density read, density and psi written
    assert h["step"] == h["collide"] + h["psi"]
    o = bench.algorithmic_bytes(Q, onepass=True)
    assert o["step"] == 2 * pop and o["psi"] == 0
    assert (Q, b["step"]) in ((19, 236), (27, 332))


def test_whole_job_rate_uses_the_slowest_rank():
    # N ranks each advance 256^3 cells for 1000 steps; the job takes as long as the slowest rank
    cells, steps, ms = 256 ** 3, 1000, 640.0
    assert bench.whole_job_mlups(4, cells, steps, ms) == pytest.approx(4 * cells * steps / (ms * 1e-3) / 1e6)


def test_committed_traffic_matches_only_its_source():
    path = os.path.join(bench.ROOT, "profiles", "collide_q19_traffic.json")
    with open(path) as fh:
        rec = json.load(fh)
    assert rec["cells"] == 256 ** 3
    assert 0.9 < rec["dram_bytes_per_launch"] / rec["algorithmic_bytes_per_launch"] < 1.1
    got = bench.committed_traffic(19)
    # either the record matches the current kernel source (traffic reported) or it is withheld
    assert got is None or got == pytest.approx(rec["dram_bytes_per_launch"])


def test_oracle_timing_aggregates_processes():
    r = bench.oracle_timing(19, budget=5.0, max_steps=1, shape=(40, 40, 40), warmup=0, procs=2)
    assert r["procs"] == 2 and len(r["mlups_per_process"]) == 2
    assert r["mlups"] == pytest.approx(sum(r["mlups_per_process"]))
    assert r["steps"] == 2
