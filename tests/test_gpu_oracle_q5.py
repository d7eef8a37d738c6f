"""3D degree 5 (theta_T = 1296) against the oracle: its region system has 34,992 unknowns,
solved by the oracle's sparse LU in the definition's order (about 1.5 minutes of host
time), so this case sits in a file of its own, after the other GPU tests."""
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


def test_3d_degree5_matches_oracle(R):
    w = dict(flux="advection", dim=3, n=(3, 3, 3), M=5, vel=(1.0, 0.7, -0.3), lo=(0.0,) * 3,
             hi=(1.0,) * 3, cfl=0.3, ic="sin")
    s = R.Solver(3, w["n"], w["M"], vel=w["vel"], cfl=w["cfl"], lo=w["lo"], hi=w["hi"])
    rng = np.random.default_rng(31)
    q = rng.standard_normal((s.cells, s.theta_s))
    s.set_state(q)
    dt = s.info()["dt"]
    W = s.predict()
    Wo = OL.predict(q, w, dt)
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    assert rel(W, Wo) < 1e-12
    s.set_state(q)
    s.step(1)
    assert rel(s.get_state(), OL.correct(q, Wo[:, :s.theta_s], w, dt)) < 1e-12
    s.close()
