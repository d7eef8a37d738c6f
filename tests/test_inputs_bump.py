"""The paper's bump initial data (eqs. adv1d, adv2d, adv3d) and its sum-factorised
projection, against the plain tensor Gauss projection of the same function (no GPU)."""
import numpy as np
import pytest

from paper_2101_01231_gb300 import inputs as I


def _w(d, n):
    return dict(dim=d, n=(n,) * d, lo=(0.0,) * d, hi=(1.0,) * d)


def test_bump_values():
    # exp(1 / (r^2 - omega^2)) inside the ball, 0 outside; e^-9 at the centre
    assert I.paper_bump(np.array([0.5])) == pytest.approx(np.exp(-9.0), rel=1e-15)
    assert I.paper_bump(np.array([0.5 + 1.0 / 3.0]))[0] == 0.0
    x = np.array([0.6])
    assert I.paper_bump(x, x, x)[0] == pytest.approx(np.exp(1.0 / (0.03 - 1.0 / 9.0)), rel=1e-14)


@pytest.mark.parametrize("d,n,nb", [(1, 12, 4), (2, 7, 3), (3, 5, 3), (3, 6, 2)])
def test_project_bump_matches_tensor_projection(d, n, nb):
    w = _w(d, n)
    got = I.project_bump(w, nb, nq=12)
    ref = I.project_tensor(lambda *xs: I.paper_bump(*xs), w, nb, nq=12)[:, 0, :]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    # cells that do not meet the ball are exactly zero in both
    assert np.count_nonzero(np.abs(got).max(axis=1)) == np.count_nonzero(np.abs(ref).max(axis=1))


def test_bump_workloads():
    for name in ("adv2d_bump_n60_q5", "adv3d_bump_n48_q5"):
        w = I.workload(name, n=(6,) * I.WORKLOADS[name]["dim"], M=1)
        q0 = I.initial_state(w)
        assert q0.shape == (6 ** w["dim"], 2 ** w["dim"])
        np.testing.assert_array_equal(q0, I.project_bump(w, 2, nq=16))
        # a = (1, ..., 1): at t = 1 the bump is back at its start
        np.testing.assert_array_equal(I.exact_coefficients(w, 1.0), I.project_bump(w, 3, nq=16))
        with pytest.raises(ValueError):
            I.exact_coefficients(w, 0.5)
