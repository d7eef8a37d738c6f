"""Pins of the nonlinear oracle (quadrature residual, QQF / quadrature Jacobians, Newton,
nonlinear correction) against independent computations."""
import numpy as np
import pytest

from oracle import error as oerr
from oracle import linear as L
from oracle import nonlinear as NL
from paper_2101_01231_gb300 import inputs as I


def _fd_jacobian(W, Q, flux, tb, lam, alpha, eps=1e-6):
    E = W.shape[0]
    Wf = W.reshape(E, -1)
    n = Wf.shape[1]
    J = np.zeros((E, n, n))
    for c in range(n):
        Wp, Wm = Wf.copy(), Wf.copy()
        Wp[:, c] += eps
        Wm[:, c] -= eps
        Rp, _ = NL.residual(Wp.reshape(W.shape), Q, flux, tb, lam, alpha)
        Rm, _ = NL.residual(Wm.reshape(W.shape), Q, flux, tb, lam, alpha)
        J[:, :, c] = (Rp - Rm).reshape(E, -1) / (2 * eps)
    return J


def test_euler_flux_jacobian_matches_finite_differences():
    fl = NL.Euler2D(1.4)
    rng = np.random.default_rng(0)
    w = np.stack([1.0 + 0.2 * rng.random(7), 0.3 * rng.standard_normal(7),
                  0.3 * rng.standard_normal(7), 2.5 + rng.random(7)])
    for dd in (0, 1):
        A = fl.dF(w, dd)
        eps = 1e-7
        for j in range(4):
            wp, wm = w.copy(), w.copy()
            wp[j] += eps
            wm[j] -= eps
            fd = (fl.F(wp, dd) - fl.F(wm, dd)) / (2 * eps)
            assert np.abs(A[:, j] - fd).max() < 1e-6


@pytest.mark.parametrize("d,M", [(1, 2), (2, 1), (2, 2), (3, 1)])
def test_burgers_qqf_equals_quadrature_and_fd(d, M):
    # F'(w) = w has degree M <= 2M, so the projection of eq. Jacproj is exact and the
    # quasi-quadrature-free Jacobian equals the quadrature one (eq. Jacobian); both
    # equal the finite-difference Jacobian of the residual with alpha held fixed.
    rng = np.random.default_rng(d * 10 + M)
    tb = NL.Tables(d, M)
    fl = NL.Burgers()
    lam = np.full(d, 0.3)
    W = 0.5 + 0.3 * rng.standard_normal((2, 3 ** d, 1, tb.thT))
    Q = rng.standard_normal((2, 3 ** d, 1, tb.thS))
    _, al = NL.residual(W, Q, fl, tb, lam)
    Jq = NL.jacobian(W, Q, fl, tb, lam, al, "qqf")
    Jd = NL.jacobian(W, Q, fl, tb, lam, al, "quad")
    scale = np.abs(Jd).max()
    assert np.abs(Jq - Jd).max() < 1e-13 * scale
    if d * M <= 3:
        Jfd = _fd_jacobian(W, Q, fl, tb, lam, al)
        assert np.abs(Jd - Jfd).max() < 1e-7 * scale


def test_euler_qqf_close_to_quadrature_jacobian():
    # For a rational flux the QQF Jacobian and the quadrature Jacobian differ by the
    # projection / quadrature error of F'(w), which vanishes for a constant state and
    # shrinks (at least quadratically) with the size of the variation.
    d, M = 2, 1
    tb = NL.Tables(d, M)
    fl = NL.Euler2D(1.4)
    lam = np.full(d, 0.1)
    gaps = []
    for amp in (1e-2, 1e-3):
        rng = np.random.default_rng(5)
        W = np.zeros((1, 9, 4, tb.thT))
        W[:, :, :, 0] = np.array([1.0, 0.5, 0.3, 2.5])
        W += amp * rng.standard_normal(W.shape)
        Q = W[..., : tb.thS].copy()
        _, al = NL.residual(W, Q, fl, tb, lam)
        Jq = NL.jacobian(W, Q, fl, tb, lam, al, "qqf")
        Jd = NL.jacobian(W, Q, fl, tb, lam, al, "quad")
        gaps.append(np.abs(Jq - Jd).max() / np.abs(Jd).max())
    assert gaps[0] < 1e-2 and gaps[1] < gaps[0] / 20
    Jfd = _fd_jacobian(W, Q, fl, tb, lam, al, eps=1e-6)
    assert np.abs(Jd - Jfd).max() < 1e-6 * np.abs(Jd).max()


def test_newton_with_linear_flux_equals_linear_prediction():
    w = dict(flux="advection", dim=2, n=(5, 4), M=2, vel=(1.0, -0.5), lo=(0, 0), hi=(1, 1), cfl=0.3)
    rng = np.random.default_rng(6)
    Q = rng.standard_normal((20, 9))
    dt = 0.03
    Wl = L.predict(Q, w, dt)
    Wn, it, cv = NL.newton_predict(Q, w, dt, return_iters=True)
    assert cv.all() and it.max() <= 2
    assert np.abs(Wl - Wn).max() < 1e-12
    assert np.abs(L.correct(Q, Wl[:, :9], w, dt) - NL.correct(Q, Wn, w, dt)).max() < 1e-13


def test_newton_converges_quadratically_for_burgers():
    w = dict(flux="burgers", dim=2, n=(8, 8), M=1, lo=(0, 0), hi=(1, 1), cfl=0.35, seed=3)
    Q = I.initial_state(w)
    dt, _ = L.time_step(w, NL.max_speed(Q, w))
    tb = NL.Tables(2, 1)
    fl = NL.Burgers()
    lam = dt / L.cell_sizes(w)
    QR = L.gather_cells(Q, w, [5]).reshape(1, 9, 1, tb.thS)
    W = np.zeros((1, 9, 1, tb.thT))
    W[..., : tb.thS] = QR
    _, al0 = NL.residual(W, QR, fl, tb, lam)
    norms = []
    for _ in range(4):
        R, al = NL.residual(W, QR, fl, tb, lam, al0)
        J = NL.jacobian(W, QR, fl, tb, lam, al0, "qqf")
        dW = np.linalg.solve(J, R.reshape(1, -1, 1)).reshape(R.shape)
        W -= dW
        norms.append(np.abs(dW).max())
    assert norms[1] < 1e-2 and norms[2] < 1e-5
    # quadratic: |d_{k+1}| <= C |d_k|^2 with a moderate C
    assert norms[2] < 10 * norms[1] ** 2 + 1e-15
    assert norms[3] < 1e-12


def test_burgers_mass_conserved_and_order():
    errs = []
    for N in (8, 16):
        w = dict(flux="burgers", dim=2, n=(N, N), M=2, lo=(0, 0), hi=(1, 1), cfl=0.35, seed=3)
        T = 0.3 * I.burgers_shock_time(w)
        Q0 = I.initial_state(w)
        dt, nt = L.time_step(w, NL.max_speed(Q0, w), T)
        Q = Q0
        for _ in range(nt):
            W, it, cv = NL.newton_predict(Q, w, dt, return_iters=True, chunk=64)
            assert cv.all()
            Q = NL.correct(Q, W, w, dt)
        h2 = 1.0 / N ** 2
        m0, m1 = Q0[:, 0].sum() * h2, Q[:, 0].sum() * h2
        assert abs(m1 - m0) < 1e-15
        errs.append(oerr.l2_relative_error(Q, I.exact_coefficients(w, T), 2, 2))
    assert oerr.observed_order(errs[0], errs[1], 1 / 8, 1 / 16) > 2.4


def test_euler_uniform_flow_is_preserved():
    w = dict(flux="euler", dim=2, n=(4, 4), M=1, lo=(0, 0), hi=(1, 1), cfl=0.3, gamma=1.4)
    Q = np.zeros((16, 4, 4))
    Q[:, :, 0] = np.array([1.2, 0.6, -0.3, 2.9])
    Q = Q.reshape(16, 16)
    dt, _ = L.time_step(w, NL.max_speed(Q, w))
    W, it, cv = NL.newton_predict(Q, w, dt, return_iters=True)
    assert cv.all()
    Q1 = NL.correct(Q, W, w, dt)
    assert np.abs(Q1 - Q).max() < 1e-13


def _burgers3d(n, M):
    w = dict(flux="burgers", dim=3, n=(n,) * 3, M=M, lo=(0.0,) * 3, hi=(1.0,) * 3, cfl=0.3)
    f = lambda x, y, z: (0.3 + 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
                         * np.sin(2 * np.pi * z) + 0.05 * np.cos(2 * np.pi * (x + z)))
    Q = I.project_tensor(f, w, M + 1)[:, 0, :]
    return w, np.ascontiguousarray(Q)


def test_newton_converges_quadratically_for_burgers_3d():
    # the 3 x 3 x 3 region of a 3D Burgers state: the QQF Newton iteration (exact Jacobian
    # for Burgers) converges quadratically, as in 2D
    w, Q = _burgers3d(4, 1)
    dt, _ = L.time_step(w, NL.max_speed(Q, w))
    tb = NL.Tables(3, 1)
    fl = NL.Burgers()
    lam = dt / L.cell_sizes(w)
    QR = L.gather_cells(Q, w, [21]).reshape(1, 27, 1, tb.thS)
    W = np.zeros((1, 27, 1, tb.thT))
    W[..., : tb.thS] = QR
    _, al0 = NL.residual(W, QR, fl, tb, lam)
    norms = []
    for _ in range(4):
        R, _ = NL.residual(W, QR, fl, tb, lam, al0)
        J = NL.jacobian(W, QR, fl, tb, lam, al0, "qqf")
        dW = np.linalg.solve(J, R.reshape(1, -1, 1)).reshape(R.shape)
        W -= dW
        norms.append(np.abs(dW).max())
    assert norms[2] < 10 * norms[1] ** 2 + 1e-15
    assert norms[3] < 1e-12


def test_burgers_3d_constant_state_and_mass():
    w, Q = _burgers3d(4, 1)
    dt, _ = L.time_step(w, NL.max_speed(Q, w))
    # a constant state is a fixed point of the prediction and of the correction
    Qc = np.zeros_like(Q)
    Qc[:, 0] = 0.4
    Wc = NL.newton_predict(Qc, w, dt)
    assert np.abs(NL.correct(Qc, Wc, w, dt) - Qc).max() < 1e-14
    # the correction conserves the mean
    W, it, cv = NL.newton_predict(Q, w, dt, return_iters=True, max_iters=8)
    assert cv.all()
    Q1 = NL.correct(Q, W, w, dt)
    assert abs(Q1[:, 0].sum() - Q[:, 0].sum()) < 1e-14 * np.abs(Q[:, 0]).sum()
