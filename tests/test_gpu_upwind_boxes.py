"""Every shape of the upwind box in 3D (velocity components zero or not, either sign): one
step of the FP64 and the mixed tensor-core path against the oracle.  The box is the set of
region cells the prediction reads: offsets {-1, 0} along a positive velocity component,
{0, +1} along a negative one, {0} along a zero one."""
import numpy as np
import pytest

from oracle import linear as OL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2101_01231_gb300 import ridg
    return ridg


VELS = [(0.0, 0.0, 0.9), (-0.7, 0.0, 0.0), (0.6, -0.8, 0.0), (0.0, 0.5, -1.0),
        (-0.4, 0.0, 0.9), (0.0, 0.0, -0.6)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("vel", VELS)
def test_3d_box_shapes_step_matches_oracle(R, vel, prec):
    w = dict(flux="advection", dim=3, n=(9, 6, 4), M=2, vel=vel, lo=(0.0,) * 3, hi=(1.0,) * 3,
             cfl=0.3, ic="sin")
    p = R.RIDG_PREC_FP64 if prec == "fp64" else R.RIDG_PREC_MIXED_BF16
    s = R.Solver(3, w["n"], w["M"], vel=w["vel"], cfl=w["cfl"], lo=w["lo"], hi=w["hi"],
                 precision=p, slices=6 if prec == "mixed" else 0)
    rng = np.random.default_rng(37)
    q = rng.standard_normal((s.cells, s.theta_s))
    s.set_state(q)
    dt = s.info()["dt"]
    s.step(1)
    ref = OL.step(q, w, dt)
    assert float(np.abs(s.get_state() - ref).max() / np.abs(ref).max()) < 1e-12
    s.close()
