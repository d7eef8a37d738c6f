"""ORACLE (test infrastructure only) -- accuracy metrics of Sec. 4.

eq. l2relerror: with X the cell-wise projection of the exact solution onto Q(M+1)
(theta_S^+ coefficients per cell) and Q the numerical Q(M) coefficients,

  error^2 = sum_i [ sum_{l in Q(M)} (X_il - Q_il)^2 + sum_{l in Q(M+1) \\ Q(M)} X_il^2 ]
            / sum_i sum_{l in Q(M+1)} X_il^2 .

eq. Mratio: observed order M ~ log(e1 / e2) / log(h1 / h2).
"""
from __future__ import annotations

import numpy as np


def modes_in(nb_small: int, nb_big: int, d: int) -> np.ndarray:
    """Boolean mask over the nb_big^d tensor modes (x fastest) of those with every
    per-dimension degree < nb_small."""
    s = np.arange(nb_big ** d)
    mi = np.stack([(s // nb_big ** k) % nb_big for k in range(d)], axis=1)
    return (mi < nb_small).all(axis=1)


def l2_relative_error(Q: np.ndarray, X: np.ndarray, M: int, d: int, m: int = 1) -> float:
    ncell = Q.shape[0]
    Qr = Q.reshape(ncell, m, (M + 1) ** d)
    Xr = X.reshape(ncell, m, (M + 2) ** d)
    inside = modes_in(M + 1, M + 2, d)
    num = ((Xr[:, :, inside] - Qr) ** 2).sum() + (Xr[:, :, ~inside] ** 2).sum()
    den = (Xr ** 2).sum()
    return float(np.sqrt(num / den))


def observed_order(e1: float, e2: float, h1: float, h2: float) -> float:
    return float(np.log(e1 / e2) / np.log(h1 / h2))
