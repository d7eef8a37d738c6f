"""ORACLE (test infrastructure only) -- RIDG for linear advection q_t + a . grad q = 0.

Prediction (Sec. 2.2, eq. pred_full_system).  On the region R_i of 3^d space-time
elements every residual is divided by |T_j| and written in reference coordinates
(x = x_j + h xi / 2, t = t^n + dt (tau + 1) / 2).  With nu_d = a_d dt / h_d and the 1D
tables D[a, b] = int phi_a' phi_b and traces phi(+-1), the pieces of eq.
pred_full_system become, per region element j and test function Psi_k = psi_alpha Phi_s:

  time term       [psi_alpha(1) psi_gamma(1) - D_{alpha gamma}] delta_{s s'}  W_j
  internal flux   - sum_d nu_d delta_{alpha gamma} (D along dim d)           W_j
  surface flux    Rusanov flux on faces interior to R_i; for linear flux it is the
                  upwind flux a+ w_L + a- w_R (a+ = max(a,0), a- = min(a,0)).
                  On the boundary of R_i only the trace internal to R_i is used
                  (F(w_int) . n), which insulates the region.
  causal source   - psi_alpha(-1) Q^n_{j, s}

The region system A W_R = B Q_R is assembled from these Kronecker factors, factored
once (it does not depend on the element on a uniform periodic mesh) and solved for every
element's region; only the centre element's W_i is kept (Sec. 2.2, fig. RIDG_2D).

Correction (Sec. 2.3): with W-bar the tau-mean (psi_0) block of W_i,
  Q^{n+1}_i = Q^n_i + sum_d nu_d (D along d) W-bar_i
              - sum_d [ phi(+1) (x)_d F_{i+1/2} - phi(-1) (x)_d F_{i-1/2} ]
where the face value F_{i+1/2} = nu+ trace_{+1}(W-bar_i) + nu- trace_{-1}(W-bar_{i+e_d})
is computed once per face and applied to both neighbours.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from . import basis


# ---------------------------------------------------------------------------
# mesh helpers
# ---------------------------------------------------------------------------
def cell_sizes(w) -> np.ndarray:
    return np.array([(w["hi"][k] - w["lo"][k]) / w["n"][k] for k in range(w["dim"])])


def grid_shape(w) -> tuple:
    """Array shape of a cell field: (n_z, n_y, n_x) truncated to the dimension."""
    return tuple(reversed(tuple(w["n"][: w["dim"]])))


def cell_axis(d: int, dd: int) -> int:
    """Axis of a (grid ...) array that runs along spatial dimension dd."""
    return d - 1 - dd


def time_step(w, max_speed: float, T: float | None = None):
    """Sec. 5 / eq. comms: dt = nu h / (max wave speed).  When a final time T is given
    the step is shortened so that an integer number of steps lands on T:
    N_t = ceil(T / dt_cfl) (with a 1e-9 guard against rounding), dt = T / N_t."""
    h = float(np.min(cell_sizes(w)))
    dt = w["cfl"] * h / max_speed
    if T is None:
        return dt, None
    nt = int(math.ceil(T / dt - 1e-9))
    return T / nt, nt


def advection_time_step(w, T=None):
    return time_step(w, float(np.max(np.abs(w["vel"][: w["dim"]]))), T)


# ---------------------------------------------------------------------------
# the region system of eq. pred_full_system
# ---------------------------------------------------------------------------
def _region_terms(d: int, M: int, nu, kron):
    """The terms of eq. pred_full_system on one region, in the order they are summed:
    yields ("A" or "B", row element, column element, block), blocks built with kron."""
    nb = M + 1
    thS = nb ** d
    D = basis.deriv_matrix(nb)
    ep, em = basis.trace_plus(nb), basis.trace_minus(nb)
    I1 = np.eye(nb)
    IS = np.eye(thS)

    def along(dd, X):  # spatial operator acting along dimension dd only
        mats = [I1] * d
        mats[dd] = X
        out = mats[-1]
        for Y in reversed(mats[:-1]):   # x index fastest
            out = kron(out, Y)
        return out

    offs = basis.region_offsets(d)
    index = {tuple(o): r for r, o in enumerate(offs)}
    time_term = np.outer(ep, ep) - D          # psi(1) psi(1)^T - int psi' psi
    source = em.reshape(nb, 1)                # psi_alpha(-1)
    for r, o in enumerate(offs):
        yield "A", r, r, kron(time_term, IS)
        yield "B", r, r, kron(source, IS)
        for dd in range(d):
            nu_d = float(nu[dd])
            nup, num = max(nu_d, 0.0), min(nu_d, 0.0)
            yield "A", r, r, -nu_d * kron(I1, along(dd, D))           # internal flux
            # face at xi_d = +1, outward normal +e_d
            o2 = o.copy(); o2[dd] += 1
            if tuple(o2) in index:
                yield "A", r, r, nup * kron(I1, along(dd, np.outer(ep, ep)))
                yield "A", r, index[tuple(o2)], num * kron(I1, along(dd, np.outer(ep, em)))
            else:   # region boundary: own (interior) trace only
                yield "A", r, r, nu_d * kron(I1, along(dd, np.outer(ep, ep)))
            # face at xi_d = -1, outward normal -e_d
            o2 = o.copy(); o2[dd] -= 1
            if tuple(o2) in index:
                yield "A", r, index[tuple(o2)], -nup * kron(I1, along(dd, np.outer(em, ep)))
                yield "A", r, r, -num * kron(I1, along(dd, np.outer(em, em)))
            else:
                yield "A", r, r, -nu_d * kron(I1, along(dd, np.outer(em, em)))


def region_system(d: int, M: int, nu) -> tuple[np.ndarray, np.ndarray]:
    """Return (A, B) with A W_R = B Q_R for one region.

    W_R stacks the 3^d space-time blocks (region element r, then alpha, then s);
    Q_R stacks the 3^d spatial blocks.  Everything is divided by |T_j|."""
    nb = M + 1
    thS = nb ** d
    thT = nb * thS
    nR = 3 ** d
    A = np.zeros((nR * thT, nR * thT))
    B = np.zeros((nR * thT, nR * thS))
    for which, r, c, blk in _region_terms(d, M, nu, np.kron):
        if which == "A":
            A[r * thT:(r + 1) * thT, c * thT:(c + 1) * thT] += blk
        else:
            B[r * thT:(r + 1) * thT, c * thS:(c + 1) * thS] += blk
    return A, B


def region_system_sparse(d: int, M: int, nu):
    """The same (A, B) as region_system, the same terms summed in the same order, stored
    as scipy sparse matrices (A in CSC for a sparse LU) -- for degrees whose dense region
    matrix does not fit (3D: 3^3 (M + 1)^4 unknowns)."""
    nb = M + 1
    thS = nb ** d
    thT = nb * thS
    nR = 3 ** d
    Ab = [[None] * nR for _ in range(nR)]
    Bb = [[None] * nR for _ in range(nR)]

    def skron(X, Y):
        return sps.kron(sps.csr_matrix(X), sps.csr_matrix(Y), format="csr")

    for which, r, c, blk in _region_terms(d, M, nu, skron):
        blocks = Ab if which == "A" else Bb
        blocks[r][c] = blk if blocks[r][c] is None else blocks[r][c] + blk
    for r in range(nR):   # bmat needs each block row and column sized
        if Bb[r][r] is None:
            Bb[r][r] = sps.csr_matrix((thT, thS))
    A = sps.bmat(Ab, format="csc")
    A.eliminate_zeros()   # terms with a zero factor (the downstream nu+- part) hold no entries
    return A, sps.bmat(Bb, format="csr")


def nu_of(w, dt) -> np.ndarray:
    return np.asarray(w["vel"][: w["dim"]], dtype=np.float64) * dt / cell_sizes(w)


# ---------------------------------------------------------------------------
# prediction and correction
# ---------------------------------------------------------------------------
def gather_region(Q: np.ndarray, w) -> np.ndarray:
    """X[e, r, :] = Q of the r-th vertex neighbour of cell e (periodic)."""
    d = w["dim"]
    g = grid_shape(w)
    Qg = Q.reshape(g + (Q.shape[-1],))
    out = []
    for o in basis.region_offsets(d):
        shifted = Qg
        for dd in range(d):
            if o[dd]:
                shifted = np.roll(shifted, -int(o[dd]), axis=cell_axis(d, dd))
        out.append(shifted.reshape(-1, Q.shape[-1]))
    return np.stack(out, axis=1)


# above this many region unknowns the dense region matrix (n^2 doubles, 2.3 GB at 3D Q4) is
# replaced by the same matrix in sparse form and a sparse LU (a library primitive)
DENSE_MAX_UNKNOWNS = 8000


def region_solver(d: int, M: int, nu):
    """(solve, B) for the region system A W_R = B Q_R: solve(rhs) returns A^-1 rhs."""
    n = 3 ** d * (M + 1) ** (d + 1)
    if n <= DENSE_MAX_UNKNOWNS:
        A, B = region_system(d, M, nu)
        lu = sla.lu_factor(A)
        return (lambda rhs: sla.lu_solve(lu, rhs)), B
    A, B = region_system_sparse(d, M, nu)
    # unknowns in the order of the definition (region element, then time, then space): the
    # matrix is block-structured by region element, and this order keeps the LU's fill
    # inside its blocks (3D Q5: 2.2e8 entries, factored in ~1.5 minutes)
    lu = spla.splu(A, permc_spec="NATURAL")
    return (lambda rhs: lu.solve(np.asarray(rhs))), B


def predict(Q: np.ndarray, w, dt: float, chunk: int = 8192) -> np.ndarray:
    """Centre-element space-time coefficients W_i for every cell, shape (cells, theta_T).
    Each region system is solved with the LU factors of A (computed once)."""
    d, M = w["dim"], w["M"]
    nb = M + 1
    thS, thT = nb ** d, nb ** (d + 1)
    solve, B = region_solver(d, M, nu_of(w, dt))
    rc = (3 ** d - 1) // 2
    ncell = Q.shape[0]
    W = np.empty((ncell, thT))
    for e0 in range(0, ncell, chunk):
        e1 = min(ncell, e0 + chunk)
        X = gather_region(Q, w)[e0:e1] if ncell <= chunk else _gather_rows(Q, w, e0, e1)
        rhs = B @ X.reshape(e1 - e0, -1).T                     # (n, cells)
        sol = solve(rhs)
        W[e0:e1] = sol[rc * thT:(rc + 1) * thT].T
    return W


def _gather_rows(Q, w, e0, e1):
    return gather_cells(Q, w, np.arange(e0, e1))


def gather_cells(Q, w, e):
    """X[c, r, :] = Q of the r-th vertex neighbour of cell e[c] (periodic)."""
    d = w["dim"]
    n = w["n"]
    e = np.asarray(e)
    idx = [(e // int(np.prod(n[:k]))) % n[k] for k in range(d)]
    cols = []
    for o in basis.region_offsets(d):
        lin = np.zeros_like(e)
        stride = 1
        for k in range(d):
            lin += ((idx[k] + int(o[k])) % n[k]) * stride
            stride *= n[k]
        cols.append(Q[lin])
    return np.stack(cols, axis=1)


def _apply_along(T, mat, axis):
    return np.moveaxis(np.tensordot(mat, T, axes=([1], [axis])), 0, axis)


def _trace_along(T, vec, axis):
    return np.tensordot(T, vec, axes=([axis], [0]))


def _outer_along(F, vec, axis):
    shape = [1] * (F.ndim + 1)
    shape[axis] = vec.size
    return np.expand_dims(F, axis) * vec.reshape(shape)


def correct(Q: np.ndarray, Wbar: np.ndarray, w, dt: float) -> np.ndarray:
    """Q^{n+1} from Q^n and the tau-mean prediction W-bar (both (cells, theta_S))."""
    d, M = w["dim"], w["M"]
    nb = M + 1
    g = grid_shape(w)
    modes = (nb,) * d
    Wg = Wbar.reshape(g + modes)
    dQ = np.zeros_like(Wg)
    D = basis.deriv_matrix(nb)
    ep, em = basis.trace_plus(nb), basis.trace_minus(nb)
    nu = nu_of(w, dt)
    for dd in range(d):
        ca = cell_axis(d, dd)
        ma = d + (d - 1 - dd)           # mode axis of dimension dd
        nup, num = max(nu[dd], 0.0), min(nu[dd], 0.0)
        dQ += nu[dd] * _apply_along(Wg, D, ma)                       # volume term
        tr_p = _trace_along(Wg, ep, ma)                              # W-bar_i at xi_d = +1
        tr_m = _trace_along(Wg, em, ma)                              # W-bar_i at xi_d = -1
        flux = nup * tr_p + num * np.roll(tr_m, -1, axis=ca)         # face i+1/2, once
        dQ -= _outer_along(flux, ep, ma)                             # outflow through +1
        dQ += _outer_along(np.roll(flux, 1, axis=ca), em, ma)        # inflow through -1
    return Q + dQ.reshape(Q.shape)


def step(Q: np.ndarray, w, dt: float) -> np.ndarray:
    nb = w["M"] + 1
    thS = nb ** w["dim"]
    W = predict(Q, w, dt)
    return correct(Q, W[:, :thS], w, dt)


def run(Q0: np.ndarray, w, dt: float, nsteps: int) -> np.ndarray:
    Q = Q0.copy()
    for _ in range(nsteps):
        Q = step(Q, w, dt)
    return Q


def mass(Q: np.ndarray, w) -> float:
    """sum_i |T_i| Q_{i,0} (the cell average is the phi_0 coefficient)."""
    nb = w["M"] + 1
    thS = nb ** w["dim"]
    vol = float(np.prod(cell_sizes(w)))
    return float(Q.reshape(Q.shape[0], -1, thS)[:, :, 0].sum(axis=0).sum() * vol)


# ---------------------------------------------------------------------------
# the same step on a sample of cells (for meshes too large to run whole)
# ---------------------------------------------------------------------------
def predict_cells(Q: np.ndarray, w, dt: float, cells) -> np.ndarray:
    """W_i (theta_T) for the listed cells only, by solving their region systems."""
    d, M = w["dim"], w["M"]
    nb = M + 1
    thT = nb ** (d + 1)
    solve, B = region_solver(d, M, nu_of(w, dt))
    rc = (3 ** d - 1) // 2
    cells = np.asarray(cells)
    X = gather_cells(Q, w, cells)
    sol = solve(B @ X.reshape(len(cells), -1).T)
    return sol[rc * thT:(rc + 1) * thT].T


def face_neighbour(w, e, dd, side):
    n = w["n"]
    d = w["dim"]
    idx = [(e // int(np.prod(n[:k]))) % n[k] for k in range(d)]
    idx[dd] = (idx[dd] + side) % n[dd]
    lin, stride = 0, 1
    for k in range(d):
        lin += idx[k] * stride
        stride *= n[k]
    return lin


def step_cells(Q: np.ndarray, w, dt: float, cells) -> np.ndarray:
    """Q^{n+1} at the listed cells: the correction of Sec. 2.3 evaluated cell by cell
    from the predictions of each cell and its 2d face neighbours."""
    d, M = w["dim"], w["M"]
    nb = M + 1
    thS = nb ** d
    cells = [int(c) for c in cells]
    need = sorted(set(cells) | {face_neighbour(w, c, dd, s) for c in cells
                                for dd in range(d) for s in (-1, 1)})
    Wn = dict(zip(need, predict_cells(Q, w, dt, need)[:, :thS]))
    D = basis.deriv_matrix(nb)
    ep, em = basis.trace_plus(nb), basis.trace_minus(nb)
    nu = nu_of(w, dt)
    out = np.empty((len(cells), thS))
    modes = (nb,) * d
    for i, c in enumerate(cells):
        Wc = Wn[c].reshape(modes)
        dq = np.zeros(modes)
        for dd in range(d):
            ma = d - 1 - dd
            nup, num = max(nu[dd], 0.0), min(nu[dd], 0.0)
            Wr = Wn[face_neighbour(w, c, dd, +1)].reshape(modes)
            Wl = Wn[face_neighbour(w, c, dd, -1)].reshape(modes)
            dq += nu[dd] * _apply_along(Wc, D, ma)
            f_right = nup * _trace_along(Wc, ep, ma) + num * _trace_along(Wr, em, ma)
            f_left = nup * _trace_along(Wl, ep, ma) + num * _trace_along(Wc, em, ma)
            dq -= _outer_along(f_right, ep, ma)
            dq += _outer_along(f_left, em, ma)
        out[i] = Q[c] + dq.reshape(-1)
    return out
