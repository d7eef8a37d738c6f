"""The mixed-precision (BF16 tensor-core, split-operand) step against the oracle."""
import json
import os

import numpy as np
import pytest

from oracle import error as oerr
from oracle import linear as OL
from paper_2101_01231_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_accuracy.json")

# 2D cases: tiles of 8 x 16 cells, so these cover partial tiles in x and y, a mesh smaller
# than one tile, both velocity signs, a zero velocity component and degrees 1..3
CASES = [
    ((12, 10), 3, (1.0, 0.5)),
    ((17, 9), 2, (0.7, -0.9)),
    ((3, 3), 1, (-0.4, 1.0)),
    ((40, 33), 3, (-1.0, -0.25)),
    ((24, 20), 3, (0.8, 0.0)),
    ((11, 18), 2, (0.0, -0.6)),
]
TOL_STEP = 1e-12
TOL_FINAL = 1e-10


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2101_01231_gb300 import ridg
    return ridg


def _w(n, M, vel, cfl=0.35):
    return dict(flux="advection", dim=2, n=tuple(n), M=M, vel=tuple(vel), lo=(0.0, 0.0),
                hi=(1.0, 1.0), cfl=cfl, ic="sin")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _mixed(R, w, slices=6):
    return R.Solver(2, w["n"], w["M"], vel=w["vel"], cfl=w["cfl"], precision=R.RIDG_PREC_MIXED_BF16,
                    slices=slices)


@pytest.mark.parametrize("n,M,vel", CASES)
def test_mixed_step_matches_oracle(R, n, M, vel):
    w = _w(n, M, vel)
    s = _mixed(R, w)
    rng = np.random.default_rng(21)
    q = rng.standard_normal((s.cells, s.theta_s))
    s.set_state(q)
    dt = s.info()["dt"]
    s.step(1)
    s.sync()
    assert _rel(s.get_state(), OL.step(q, w, dt)) < TOL_STEP
    s.close()


@pytest.mark.parametrize("n,M,vel", CASES[:3])
def test_mixed_prediction_matches_oracle(R, n, M, vel):
    w = _w(n, M, vel)
    s = _mixed(R, w)
    rng = np.random.default_rng(22)
    q = rng.standard_normal((s.cells, s.theta_s))
    s.set_state(q)
    dt = s.info()["dt"]
    W = s.predict()
    s.sync()
    assert _rel(W, OL.predict(q, w, dt)) < TOL_STEP
    s.close()


def test_mixed_scale_invariance_and_zero_state(R):
    # the per-tile exponent makes the result independent of the overall scale, and an
    # all-zero state (no exponent) stays exactly zero
    w = _w((16, 16), 3, (1.0, 0.5))
    s = _mixed(R, w)
    rng = np.random.default_rng(23)
    q = rng.standard_normal((s.cells, s.theta_s))
    outs = []
    for scale in (1.0, 2.0 ** -300, 2.0 ** 300):
        s.set_state(q * scale)
        s.step(1)
        s.sync()
        outs.append(s.get_state() / scale)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    s.set_state(np.zeros_like(q))
    s.step(3)
    assert not np.any(s.get_state())
    s.close()


def test_mixed_mass_conserved(R):
    w = _w((40, 33), 3, (1.0, 0.5))
    s = _mixed(R, w)
    q = np.random.default_rng(24).standard_normal((s.cells, s.theta_s)) + 2.0
    s.set_state(q)
    m0 = s.mass()[0]
    s.step(50)
    s.sync()
    assert abs(s.mass()[0] - m0) <= 4e-14 * abs(m0)
    s.close()


def test_mixed_final_time_parity(R):
    w = I.workload("adv2d_n256_q3", n=(48, 40))
    s = _mixed(R, w)
    q0 = I.initial_state(w)
    s.set_state(q0)
    nt = s.set_final_time(0.25)
    s.step(nt)
    s.sync()
    dt, nt_o = OL.advection_time_step(w, T=0.25)
    assert nt == nt_o
    assert _rel(s.get_state(), OL.run(q0, w, dt, nt)) < TOL_FINAL
    s.close()


def test_mixed_error_decreases_with_slices(R):
    w = _w((24, 24), 3, (1.0, 0.5))
    rng = np.random.default_rng(25)
    q = rng.standard_normal((24 * 24, 16))
    errs = []
    for S in (2, 3, 4, 5, 6):
        s = _mixed(R, w, slices=S)
        s.set_state(q)
        dt = s.info()["dt"]
        s.step(1)
        s.sync()
        errs.append(_rel(s.get_state(), OL.step(q, w, dt)))
        s.close()
    for a, b in zip(errs, errs[1:]):
        assert b < a or b < 1e-15, errs
    assert errs[0] > 1e-6 and errs[-1] < 1e-12, errs


def test_mixed_equal_accuracy_on_full_workload(R):
    """256 x 256, Q3, to t = 1 (732 steps): the mixed path's L2 error against the exact
    solution is within 1.05x of the oracle's (the oracle's figure is stored by
    tests/golden/make_golden.py)."""
    gold = json.load(open(GOLDEN)).get("adv2d_n256_q3")
    if gold is None:
        pytest.skip("oracle accuracy figure not generated")
    w = I.workload("adv2d_n256_q3")
    s = _mixed(R, w)
    s.set_state(I.initial_state(w))
    nt = s.set_final_time(1.0)
    assert nt == gold["steps"]
    s.step(nt)
    s.sync()
    e = s.l2_error(I.exact_coefficients(w, 1.0))
    assert e <= 1.05 * gold["l2_error"], (e, gold["l2_error"])
    s.close()


@pytest.mark.parametrize("dim,n,M,vel", [(2, (16, 13), 3, (1.0, 0.5)),
                                         (3, (10, 17, 3), 2, (1.0, 0.7, 0.3))])
def test_fp16_digits_are_bit_identical_to_bf16(R, dim, n, M, vel):
    # the balanced base-256 digits are exact in FP16 as in BF16, and every digit product and
    # FP32 sum is the same: the two operand types give the same bits (prediction and steps)
    w = dict(flux="advection", dim=dim, n=n, M=M, vel=vel, lo=(0.0,) * dim, hi=(1.0,) * dim,
             cfl=0.3, ic="sin")
    q = np.random.default_rng(41).standard_normal((int(np.prod(n)), (M + 1) ** dim))
    out = {}
    for prec in (R.RIDG_PREC_MIXED_BF16, R.RIDG_PREC_MIXED_FP16):
        s = R.Solver(dim, n, M, vel=vel, cfl=0.3, precision=prec, slices=4)
        s.set_state(q)
        W = s.predict()
        s.set_state(q)
        s.step(3)
        s.sync()
        out[prec] = (W, s.get_state())
        s.close()
    for a, b in zip(out[R.RIDG_PREC_MIXED_BF16], out[R.RIDG_PREC_MIXED_FP16]):
        assert np.array_equal(a, b)
