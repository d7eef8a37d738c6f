"""The exact L2 error of a translated piecewise polynomial (inputs.shifted_polynomial_error):
the error measure of the noisy 3D workload, whose exact solution is its piecewise
polynomial initial data carried by a t (cut by the mesh into 2^d sub-boxes per cell)."""
import numpy as np

from oracle import error as oerr
from paper_2101_01231_gb300 import inputs as I


def _w(n, vel, M=2):
    return dict(flux="advection", dim=len(n), n=tuple(n), M=M, vel=tuple(vel),
                lo=(0.0,) * len(n), hi=(1.0,) * len(n))


def test_whole_cell_shift_equals_the_projection_formula():
    # a shift by whole cells keeps the exact solution in Q(M): eq. l2relerror is then exact
    rng = np.random.default_rng(0)
    n = (6, 5, 4)
    w = _w(n, (2 / 6, 1 / 5, 3 / 4))        # shifts of 2, 1, 3 cells at t = 1
    Q0 = rng.standard_normal((120, 27))
    Q = Q0 + 1e-3 * rng.standard_normal(Q0.shape)
    B = np.roll(Q0.reshape(4, 5, 6, 27), shift=(3, 1, 2), axis=(0, 1, 2)).reshape(120, 27)
    X = np.zeros((120, 64))
    X[:, oerr.modes_in(3, 4, 3)] = B
    e = I.shifted_polynomial_error(w, Q0, Q, 1.0)
    assert abs(e - oerr.l2_relative_error(Q, X, 2, 3)) < 1e-13
    assert I.shifted_polynomial_error(w, Q0, B, 1.0) < 1e-15


def test_fractional_shift_matches_a_fine_sampling():
    # discontinuous integrand: the midpoint sum on 240^3 points converges to it (~0.1 %)
    rng = np.random.default_rng(1)
    w = _w((3, 3, 3), (0.37, 0.71, 0.13))
    Q0, Q = rng.standard_normal((27, 27)), rng.standard_normal((27, 27))
    e = I.shifted_polynomial_error(w, Q0, Q, 1.0)

    def ev(C, x, y, z):
        idx = [np.floor(v * 3).astype(int) % 3 for v in (x, y, z)]
        xi = [2 * (v * 3 - np.floor(v * 3)) - 1 for v in (x, y, z)]
        V = [I._legendre_orthonormal(3, v) for v in xi]
        c = C.reshape(3, 3, 3, 3, 3, 3)[idx[2], idx[1], idx[0]]
        return np.einsum("...cba,c...,b...,a...->...", c, V[2], V[1], V[0])

    g = (np.arange(240) + 0.5) / 240
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    num = ((ev(Q, X, Y, Z) - ev(Q0, (X - 0.37) % 1, (Y - 0.71) % 1, (Z - 0.13) % 1)) ** 2).mean()
    ref = np.sqrt(num / (Q0 ** 2).sum() * 27)
    assert abs(e - ref) < 2e-3 * ref, (e, ref)


def test_smooth_data_agrees_with_the_projection_formula():
    # for smooth data on a fine mesh the two error measures agree to leading order
    w = I.workload("adv3d_n96_q2", n=(16, 16, 16), ic="sin")
    Q0 = I.initial_state(w)
    t = 0.37
    Q = I.exact_coefficients(w, t, nb=3)          # the exact solution's Q(M) projection
    e = I.shifted_polynomial_error(w, Q0, Q, t)
    ep = oerr.l2_relative_error(Q0, I.exact_coefficients(w, 0.0), 2, 3)
    # Q0 itself carries the projection error, which the shifted exact solution inherits
    # and the Q(M) projection at t removes again: the two differ by about sqrt(2)
    assert 0.5 * ep < e < 3 * ep, (e, ep)
