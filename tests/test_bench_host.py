"""The benchmark's host-side accounting on CPU: the count of upwind region cells the linear
prediction reads (its algorithmic work) and the sampled oracle step estimate."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2101_01231_gb300 import inputs as I  # noqa: E402


def test_upwind_cells():
    assert bench.upwind_cells(dict(dim=2, vel=(1.0, 0.5))) == 4
    assert bench.upwind_cells(dict(dim=3, vel=(1.0, -0.7, 0.3))) == 8
    assert bench.upwind_cells(dict(dim=2, vel=(0.0, -0.4))) == 2
    assert bench.upwind_cells(dict(dim=1, vel=(0.0, 5.0))) == 1


def test_sampled_oracle_step_estimate():
    w = dict(name="adv3d_small", flux="advection", dim=3, n=(6, 5, 4), M=1,
             vel=(1.0, 0.7, -0.3), lo=(0.0,) * 3, hi=(1.0,) * 3, cfl=0.3, ic="sin")
    q = np.random.default_rng(0).standard_normal((120, 8))
    r = bench.cpu_oracle_sampled(w, q, nsample=16)
    assert r["kind"] == "oracle" and r["unit"] == "element-DOF updates/s"
    assert r["value"] > 0 and r["extrapolated_step_s"] > 0
    assert "16 seeded cells" in r["sample"]
