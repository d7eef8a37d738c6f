"""ORACLE (test infrastructure only) -- 1D tables for the RIDG discretisation.

Sec. 2.1: the spatial basis Phi is orthonormal with respect to the element average,
(1/|T|) int_T Phi_k Phi_l = delta_kl; on a Cartesian cell it is the tensor product of
phi_b(xi) = sqrt(2b+1) P_b(xi), xi in [-1, 1].  The space-time basis Psi of Sec. 2.2
is the same construction with one more (time) factor psi_a(tau), tau in [-1, 1].

Everything here is evaluated from numpy's Legendre series routines and Gauss-Legendre
rules (library primitives); the tables are then plain quadratures of products.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg


def gauss(n: int):
    """Gauss-Legendre nodes and weights on [-1, 1] (exact to degree 2n-1)."""
    return npleg.leggauss(n)


def _series(b: int) -> np.ndarray:
    c = np.zeros(b + 1)
    c[b] = 1.0
    return c


def phi(nb: int, x) -> np.ndarray:
    """V[b, ...] = phi_b(x) = sqrt(2b+1) P_b(x), b = 0 .. nb-1."""
    x = np.asarray(x, dtype=np.float64)
    return np.stack([math.sqrt(2 * b + 1) * npleg.legval(x, _series(b)) for b in range(nb)])


def dphi(nb: int, x) -> np.ndarray:
    """V[b, ...] = phi_b'(x)."""
    x = np.asarray(x, dtype=np.float64)
    return np.stack([math.sqrt(2 * b + 1) * npleg.legval(x, npleg.legder(_series(b)))
                     for b in range(nb)])


def trace_plus(nb: int) -> np.ndarray:
    """phi_b(+1)."""
    return phi(nb, np.array(1.0)).reshape(nb)


def trace_minus(nb: int) -> np.ndarray:
    """phi_b(-1)."""
    return phi(nb, np.array(-1.0)).reshape(nb)


def deriv_matrix(nb: int) -> np.ndarray:
    """D[a, b] = int_{-1}^{1} phi_a'(x) phi_b(x) dx (exact Gauss quadrature)."""
    x, w = gauss(nb + 1)
    return np.einsum("aq,bq,q->ab", dphi(nb, x), phi(nb, x), w)


def mass_matrix(nb: int) -> np.ndarray:
    """int phi_a phi_b dx = 2 delta_ab (computed, not assumed)."""
    x, w = gauss(nb + 1)
    V = phi(nb, x)
    return np.einsum("aq,bq,q->ab", V, V, w)


def triple(na: int, nb: int, nc: int, deriv_first: bool = False) -> np.ndarray:
    """T[a, b, c] = int_{-1}^{1} f_a phi_b phi_c dx with f = phi (or phi' when
    deriv_first) -- the 1D factors of the precomputed integrals of eq. Jacobian2."""
    n = (na + nb + nc) // 2 + 2
    x, w = gauss(n)
    F = dphi(na, x) if deriv_first else phi(na, x)
    return np.einsum("aq,bq,cq,q->abc", F, phi(nb, x), phi(nc, x), w)


# --- tensor-index helpers (x fastest; time slowest in space-time indices) ---------
def kron_x_fastest(mats):
    """Kronecker product of per-dimension factors [A_x, A_y, A_z] with the x index
    varying fastest in the combined index."""
    out = mats[-1]
    for A in reversed(mats[:-1]):
        out = np.kron(out, A)
    return out


def multi_index(nb: int, d: int) -> np.ndarray:
    """mi[s] = (b_x, b_y, b_z) of the spatial mode s = b_x + nb b_y + nb^2 b_z."""
    s = np.arange(nb ** d)
    return np.stack([(s // nb ** k) % nb for k in range(d)], axis=1)


def region_offsets(d: int) -> np.ndarray:
    """The 3^d vertex-neighbour offsets of a region (eq. region), x fastest."""
    return multi_index(3, d) - 1
