"""The 3D nonlinear prediction (NEXT-3): Burgers' flux on 3 x 3 x 3 regions, Newton with the
quasi-quadrature-free Jacobian and a dense per-region LU, and the quadrature correction,
through the C ABI against the oracle (whose 3D Newton and QQF Jacobian are pinned on the
CPU: QQF = quadrature = finite-difference Jacobian, quadratic convergence, constants kept,
mass conserved)."""
import numpy as np
import pytest

from oracle import linear as OL
from oracle import nonlinear as NL
from paper_2101_01231_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2101_01231_gb300 import ridg
    return ridg


def _w(n):
    return dict(flux="burgers", dim=3, n=tuple(n), M=1, lo=(0.0,) * 3, hi=(1.0,) * 3, cfl=0.3)


def _state(w):
    f = lambda x, y, z: (0.3 + 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
                         * np.sin(2 * np.pi * z) + 0.05 * np.cos(2 * np.pi * (x + z)))
    return np.ascontiguousarray(I.project_tensor(f, w, 2)[:, 0, :])


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-9)])
def test_3d_burgers_prediction_and_step_match_oracle(R, prec, tol):
    w = _w((4, 4, 3))
    q = _state(w)
    p = {"fp64": R.RIDG_PREC_FP64, "fp32": R.RIDG_PREC_MIXED_FP32}[prec]
    # (one of these regions needs 5 iterations, in the oracle too: cap 8 on both sides)
    s = R.Solver(3, w["n"], 1, flux="burgers", cfl=w["cfl"], precision=p, newton_max_iters=8)
    s.set_state(q)
    dt = s.info()["dt"]
    dt_or, _ = OL.time_step(w, NL.max_speed(q, w))
    assert abs(dt - dt_or) <= 1e-14 * dt_or
    W = s.predict()
    info = s.info()
    assert info["newton_unconverged"] == 0
    Wo, it, cv = NL.newton_predict(q, w, dt, return_iters=True, max_iters=8)
    assert cv.all()
    assert _rel(W, Wo) < tol
    if prec == "fp64":
        assert info["newton_iters_max"] == it.max()   # the oracle's iteration path
    s.correct()
    q1 = s.get_state()
    assert _rel(q1, NL.correct(q, Wo, w, dt)) < tol
    # the correction conserves the mean to round-off
    assert abs(q1[:, 0].sum() - q[:, 0].sum()) <= 1e-14 * np.abs(q[:, 0]).sum()
    s.close()


def test_3d_burgers_constant_state_and_graph_steps(R):
    w = _w((5, 3, 4))
    s = R.Solver(3, w["n"], 1, flux="burgers", cfl=w["cfl"], newton_max_iters=8)
    qc = np.zeros((60, 8))
    qc[:, 0] = 0.4
    s.set_state(qc)
    s.step(2)
    assert s.sync() == R.RIDG_OK
    assert np.abs(s.get_state() - qc).max() < 1e-14     # a constant is a fixed point
    # two captured steps equal two oracle steps
    q = _state(w)
    s.set_state(q)
    dt = s.info()["dt"]
    s.step(2)
    assert s.sync() == R.RIDG_OK
    q2 = NL.step(NL.step(q, w, dt, max_iters=8), w, dt, max_iters=8)
    assert _rel(s.get_state(), q2) < 1e-12
    s.close()


def test_3d_nonlinear_rejects_unsupported(R):
    with pytest.raises(R.RidgError):
        R.Solver(3, (4, 4, 4), 2, flux="burgers")        # degree 2: not built in 3D
    with pytest.raises(R.RidgError):
        R.Solver(3, (4, 4, 4), 1, flux="euler")          # Euler is 2D
    with pytest.raises(R.RidgError):
        R.Solver(3, (4, 4, 4), 1, flux="burgers", precision=R.RIDG_PREC_MIXED_TF32)
