"""Pins of the oracle's 1D tables against closed forms (no GPU)."""
import math

import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_gauss_exact_to_degree_2n_minus_1(n):
    x, w = basis.gauss(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("nb", [1, 2, 4, 7, 12])
def test_orthonormal_in_average_sense(nb):
    # (1/2) int phi_a phi_b = delta_ab  (Sec. 2.1 normalisation)
    assert np.allclose(0.5 * basis.mass_matrix(nb), np.eye(nb), atol=1e-13)


def test_traces_closed_form():
    # P_n(+-1) = (+-1)^n  =>  phi_b(+-1) = (+-1)^b sqrt(2b+1)
    nb = 10
    b = np.arange(nb)
    assert np.allclose(basis.trace_plus(nb), np.sqrt(2 * b + 1), atol=1e-13)
    assert np.allclose(basis.trace_minus(nb), (-1.0) ** b * np.sqrt(2 * b + 1), atol=1e-13)


def test_derivative_matrix_closed_form():
    # int P_a' P_b = 2 iff a > b and a + b odd, else 0
    nb = 9
    D = basis.deriv_matrix(nb)
    for a in range(nb):
        for b in range(nb):
            ref = 2.0 if (a > b and (a + b) % 2 == 1) else 0.0
            ref *= math.sqrt((2 * a + 1) * (2 * b + 1))
            assert abs(D[a, b] - ref) < 1e-12


def _gaunt(a, b, c):
    """int_{-1}^{1} P_a P_b P_c = 2 (a b c; 0 0 0)^2 (closed form of the 3j symbol)."""
    if (a + b + c) % 2 or a > b + c or b > a + c or c > a + b:
        return 0.0
    s = (a + b + c) // 2
    f = math.factorial
    w = (f(2 * s - 2 * a) * f(2 * s - 2 * b) * f(2 * s - 2 * c) / f(2 * s + 1)) * (
        f(s) / (f(s - a) * f(s - b) * f(s - c))) ** 2
    return 2.0 * w


def test_triple_products_closed_form():
    na, nb, nc = 5, 5, 9
    T = basis.triple(na, nb, nc)
    for a in range(na):
        for b in range(nb):
            for c in range(nc):
                ref = _gaunt(a, b, c) * math.sqrt((2 * a + 1) * (2 * b + 1) * (2 * c + 1))
                assert abs(T[a, b, c] - ref) < 1e-12


def test_derivative_triple_products_by_parts():
    # int phi_a' phi_b phi_c = [phi_a phi_b phi_c]_{-1}^{1} - int phi_a (phi_b phi_c)'
    nb, nc = 4, 7
    T1 = basis.triple(nb, nb, nc, deriv_first=True)
    x, w = basis.gauss(12)
    V = {n: basis.phi(n, x) for n in (nb, nc)}
    dV = {n: basis.dphi(n, x) for n in (nb, nc)}
    ep = {n: basis.trace_plus(n) for n in (nb, nc)}
    em = {n: basis.trace_minus(n) for n in (nb, nc)}
    bnd = np.einsum("a,b,c->abc", ep[nb], ep[nb], ep[nc]) - np.einsum("a,b,c->abc", em[nb], em[nb], em[nc])
    inner = np.einsum("aq,bq,cq,q->abc", V[nb], dV[nb], V[nc], w) + np.einsum(
        "aq,bq,cq,q->abc", V[nb], V[nb], dV[nc], w)
    assert np.allclose(T1, bnd - inner, atol=1e-12)


def test_kron_x_fastest_ordering():
    mi = basis.multi_index(3, 3)
    A = [np.diag([1.0, 2.0, 3.0]), np.diag([10.0, 20.0, 30.0]), np.diag([100.0, 200.0, 300.0])]
    K = np.diag(basis.kron_x_fastest(A))
    assert np.allclose(K, (mi[:, 0] + 1) * 10 * (mi[:, 1] + 1) * 100 * (mi[:, 2] + 1))
    offs = basis.region_offsets(2)
    assert offs.shape == (9, 2) and tuple(offs[4]) == (0, 0) and tuple(offs[1]) == (0, -1)
