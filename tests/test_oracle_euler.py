"""Pins of the oracle's compressible Euler flux (oracle/nonlinear.py, Euler2D) against what
the physics fixes, independently of the flux's own formulas:

* the characteristic speeds: the eigenvalues of dF_d/dq, taken by central differences of
  the oracle's F, are u_d - c, u_d, u_d, u_d + c with c = sqrt(gamma p / rho) for a state
  built from primitive variables (ideal-gas total energy E = p / (gamma - 1) + rho |u|^2 / 2),
  and speed() is the largest of their magnitudes;
* the spatial DG operator of the correction (Sec. 2.3, Rusanov faces) applied to the
  projected isentropic vortex converges to the projection of its exact time derivative
  (the vortex translates with the ambient velocity (1, 1)) at the order M of a DG
  truncation error, on 16^2, 32^2, 64^2 meshes, degrees 1 and 2;
* whole RIDG steps of the oracle (Newton prediction + correction) on the vortex converge
  to the translated vortex at order M + 1 (eq. l2relerror, eq. Mratio).
A wrong pressure law, a dropped pressure work term or a swapped momentum flux leaves an
O(1) error in the operator test (it stagnates near 0.2 instead of falling).
"""
import multiprocessing as mp

import numpy as np
import pytest

from oracle import error as oerr
from oracle import linear as L
from oracle import nonlinear as NL
from paper_2101_01231_gb300 import inputs as I


def _fd_jacobian(f, q, h=1e-6):
    J = np.zeros((4, 4))
    for k in range(4):
        dq = np.zeros(4)
        dq[k] = h * max(1.0, abs(q[k]))
        J[:, k] = (f(q + dq) - f(q - dq)) / (2 * dq[k])
    return J


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_euler_characteristic_speeds_are_u_pm_c(gamma):
    rng = np.random.default_rng(7)
    fl = NL.Euler2D(gamma)
    for _ in range(25):
        rho = rng.uniform(0.3, 3.0)
        u, v = rng.uniform(-2.0, 2.0, 2)
        p = rng.uniform(0.2, 4.0)
        q = np.array([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])
        c = np.sqrt(gamma * p / rho)
        for dd, un in ((0, u), (1, v)):
            J = _fd_jacobian(lambda s: fl.F(s[:, None], dd)[:, 0], q)
            ev = np.sort(np.linalg.eigvals(J).real)
            assert np.allclose(ev, np.sort([un - c, un, un, un + c]), atol=2e-6), (ev, un, c)
            assert abs(fl.speed(q[:, None], dd)[0] - np.abs(ev).max()) < 2e-6


def _operator_error(n, M, d=1e-4):
    w = I.workload("euler2d_n512_q2", n=(n, n), M=M)
    nb = M + 1
    Q = I.exact_coefficients(w, 0.0, nb=nb)
    W = np.zeros((Q.shape[0], 4, nb ** 3))
    W[:, :, : nb ** 2] = Q.reshape(-1, 4, nb ** 2)   # constant in time: correction = Q + dt L(Q)
    Lh = NL.correct(Q, W.reshape(len(Q), -1), w, 1.0) - Q
    Qt = (I.exact_coefficients(w, d, nb=nb) - I.exact_coefficients(w, -d, nb=nb)) / (2 * d)
    return np.linalg.norm(Lh - Qt) / np.linalg.norm(Qt)


@pytest.mark.parametrize("M", [1, 2])
def test_euler_dg_operator_converges_to_the_vortex_time_derivative(M):
    errs = [_operator_error(n, M) for n in (16, 32, 64)]
    orders = [oerr.observed_order(errs[i], errs[i + 1], 2.0, 1.0) for i in range(2)]
    assert min(orders) > M - 0.15, (errs, orders)
    assert errs[-1] < (0.2 if M == 1 else 0.01), errs


def test_euler_vortex_ridg_steps_converge_at_order_m_plus_1():
    from oracle_pool import Pool
    T, errs = 0.5, []
    with Pool() as pool:
        for n in (16, 32):
            w = I.workload("euler2d_n512_q2", n=(n, n), M=1)
            Q0 = I.initial_state(w)
            dt, nt = L.time_step(w, NL.max_speed(Q0, w), T)
            Q, _ = pool.run(Q0, w, dt, nt)
            errs.append(oerr.l2_relative_error(Q, I.exact_coefficients(w, T), 1, 2, m=4))
    order = oerr.observed_order(errs[0], errs[1], 2.0, 1.0)
    assert order > 1.8 and errs[1] < 2e-3, (errs, order)
