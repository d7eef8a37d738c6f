"""ORACLE (test infrastructure only) -- RIDG with a general (nonlinear) flux.

Residual (eq. pred_full_system), evaluated by tensor Gauss quadrature with
n_q = ceil((3M+1)/2) points per dimension (exact for a quadratic flux), divided by |T_j|,
in reference coordinates; lambda_d = dt / h_d:

  R_{j,k} = [psi_a(1) psi_g(1) - int psi_a' psi_g] W_j                       (time term)
          - lambda_d / 2^d  sum_q w_q  d_d Psi_k(q) F_d(w_j(q))             (internal flux)
          + lambda_d / 2^d  sum_{q on face} w_q Psi_k(q) (F-hat . n)(q)       (surface flux)
          - psi_a(-1) Q^n_{j,s}                                             (causal source)

Faces interior to the region use the Rusanov flux
F-hat(w_L, w_R) = (F(w_L) + F(w_R)) / 2 - alpha (w_R - w_L) / 2 with alpha the largest
wave speed |lambda(w_L)|, |lambda(w_R)| over the face's quadrature points; in the
prediction alpha is evaluated once, from the initial iterate (Q^n extended in time), and
held fixed during the Newton iteration (alpha="frozen", the reading the CUDA path
implements).  Two other readings of Sec. 2.2 are available for comparison:
alpha="live" re-evaluates the per-face alpha from every iterate in the residual (the
Jacobian then holds that iterate's alpha fixed, so Newton converges linearly), and
alpha="point" does the same with alpha taken pointwise at each face quadrature point.
Faces on the region boundary use the interior trace only, F(w_int) . n.

Jacobian (Sec. 3).  Newton W <- W - J^{-1} R (Sec. 3).  Two Jacobians are provided:
  * quadrature (eq. Jacobian): every integral int d Psi_k Psi_l F'(w) by quadrature;
  * quasi-quadrature-free (eqs. Jacproj, Jacobian2): F'(w) is projected onto Psi_p,
    p in Q(2M, d+1), with 2M+1 Gauss points per dimension, and contracted with the
    precomputed products of 1D triple-product integrals; the surface blocks project the
    Rusanov flux Jacobian (F'(w) +- alpha I)/2 (alpha fixed) onto the face basis the
    same way.  The time blocks are constant.
Newton starts from Q^n extended constant in time on every region element, stops when
||dW||_inf <= tol * max(1, ||W||_inf) or after max_iters iterations.

Correction (Sec. 2.3) uses the same quadrature with the predicted W of the cell and of its
face neighbours; every face flux is evaluated once and applied to both sides.
"""
from __future__ import annotations

import math

import numpy as np

from . import basis
from .linear import cell_sizes, grid_shape, cell_axis


# ---------------------------------------------------------------------------
# flux models
# ---------------------------------------------------------------------------
class Advection:
    """F_d(q) = a_d q (m = 1)."""

    m = 1

    def __init__(self, vel):
        self.a = np.asarray(vel, dtype=np.float64)

    def F(self, w, dd):
        return self.a[dd] * w

    def dF(self, w, dd):
        return np.full((1, 1) + w.shape[1:], self.a[dd])

    def speed(self, w, dd):
        return np.full(w.shape[1:], abs(self.a[dd]))


class Burgers:
    """F_d(q) = q^2 / 2 in every direction (eq. burger2d)."""

    m = 1

    def F(self, w, dd):
        return 0.5 * w * w

    def dF(self, w, dd):
        return w[None]

    def speed(self, w, dd):
        return np.abs(w[0])


class Euler2D:
    """Compressible Euler in 2D, conserved (rho, rho u, rho v, E), ideal gas."""

    m = 4

    def __init__(self, gamma=1.4):
        self.g = float(gamma)

    def _prim(self, w):
        rho, mx, my, E = w
        u, v = mx / rho, my / rho
        p = (self.g - 1.0) * (E - 0.5 * rho * (u * u + v * v))
        return rho, u, v, E, p

    def F(self, w, dd):
        rho, u, v, E, p = self._prim(w)
        if dd == 0:
            return np.stack([rho * u, rho * u * u + p, rho * u * v, u * (E + p)])
        return np.stack([rho * v, rho * u * v, rho * v * v + p, v * (E + p)])

    def dF(self, w, dd):
        g = self.g
        g1 = g - 1.0
        rho, u, v, E, p = self._prim(w)
        q2 = u * u + v * v
        H = (E + p) / rho
        z, o = np.zeros_like(u), np.ones_like(u)
        if dd == 0:
            rows = [[z, o, z, z],
                    [0.5 * g1 * q2 - u * u, (3.0 - g) * u, -g1 * v, g1 * o],
                    [-u * v, v, u, z],
                    [u * (0.5 * g1 * q2 - H), H - g1 * u * u, -g1 * u * v, g * u]]
        else:
            rows = [[z, z, o, z],
                    [-u * v, v, u, z],
                    [0.5 * g1 * q2 - v * v, -g1 * u, (3.0 - g) * v, g1 * o],
                    [v * (0.5 * g1 * q2 - H), -g1 * u * v, H - g1 * v * v, g * v]]
        return np.stack([np.stack(r) for r in rows])

    def speed(self, w, dd):
        rho, u, v, E, p = self._prim(w)
        c = np.sqrt(self.g * p / rho)
        return np.abs(u if dd == 0 else v) + c


def flux_model(w):
    if w["flux"] == "advection":
        return Advection(w["vel"][: w["dim"]])
    if w["flux"] == "burgers":
        return Burgers()
    if w["flux"] == "euler":
        return Euler2D(w.get("gamma", 1.4))
    raise ValueError(w["flux"])


# ---------------------------------------------------------------------------
# quadrature / projection tables
# ---------------------------------------------------------------------------
def _kron3(A, B):
    """Kronecker product of two 3-index tensors (A's indices slower)."""
    a = np.einsum("ijk,lmn->iljmkn", A, B)
    s = a.shape
    return a.reshape(s[0] * s[1], s[2] * s[3], s[4] * s[5])


class Tables:
    """Basis values at quadrature / projection points for dimension d, degree M."""

    def __init__(self, d: int, M: int, nq: int | None = None):
        self.d, self.M = d, M
        nb = self.nb = M + 1
        self.thS, self.thT = nb ** d, nb ** (d + 1)
        self.nq = nq or math.ceil((3 * M + 1) / 2)
        x, wq = basis.gauss(self.nq)
        V, dV = basis.phi(nb, x), basis.dphi(nb, x)
        kx = basis.kron_x_fastest
        # volume quadrature (tau slowest, then z, y, x)
        self.wV = np.kron(wq, kx([wq] * d))
        self.PsiV = np.kron(V, kx([V] * d))
        self.PhiV = np.kron(np.ones((1, self.nq)), kx([V] * d))      # Phi_s at (tau, xi)
        self.dPsiV, self.dPhiV = [], []
        for dd in range(d):
            f = [V] * d
            f[dd] = dV
            self.dPsiV.append(np.kron(V, kx(f)))
            self.dPhiV.append(np.kron(np.ones((1, self.nq)), kx(f)))
        # faces: (dd, side) -> values of Psi_k / Phi_s at the face points
        ep, em = basis.trace_plus(nb), basis.trace_minus(nb)
        one = np.ones(1)
        self.wF, self.PsiF, self.PhiF = [], [], []
        for dd in range(d):
            wf = [wq] * d
            wf[dd] = one
            self.wF.append(np.kron(wq, kx(wf)))
            ps, ph = {}, {}
            for side, tr in ((+1, ep), (-1, em)):
                f = [V] * d
                f[dd] = tr.reshape(nb, 1)
                ps[side] = np.kron(V, kx(f))
                ph[side] = np.kron(np.ones((1, self.nq)), kx(f))
            self.PsiF.append(ps)
            self.PhiF.append(ph)
        # time term and causal source (exact 1D tables)
        D = basis.deriv_matrix(nb)
        self.time_term = np.kron(np.outer(ep, ep) - D, np.eye(self.thS))
        self.source = np.kron(em.reshape(nb, 1), np.eye(self.thS))   # (thT, thS)
        # --- projection (quasi-quadrature-free) ---
        nbp = self.nbp = 2 * M + 1
        xp, wp = basis.gauss(nbp)
        Vp = basis.phi(nbp, xp)        # projection basis at projection points
        Vs = basis.phi(nb, xp)         # solution basis at projection points
        self.wP = np.kron(wp, kx([wp] * d))
        self.PsiP = np.kron(Vp, kx([Vp] * d))            # (nP, qP)
        self.PsiAtP = np.kron(Vs, kx([Vs] * d))          # (thT, qP)
        T0 = basis.triple(nb, nb, nbp)
        T1 = basis.triple(nb, nb, nbp, deriv_first=True)
        self.beta = []
        for dd in range(d):
            fac = [T0] * d
            fac[dd] = T1
            sp = fac[-1]
            for F in reversed(fac[:-1]):
                sp = _kron3(sp, F)
            self.beta.append(_kron3(T0, sp))            # (thT, thT, nP)
        self.wFP, self.PsiFP, self.PsiAtFP, self.gamma = [], [], [], []
        for dd in range(d):
            wf = [wp] * d
            wf[dd] = one
            self.wFP.append(np.kron(wp, kx(wf)))
            fp = [Vp] * d
            fp[dd] = np.ones((1, 1))
            self.PsiFP.append(np.kron(Vp, kx(fp)))      # face basis at face proj. points
            at, ga = {}, {}
            for side, tr in ((+1, ep), (-1, em)):
                f = [Vs] * d
                f[dd] = tr.reshape(nb, 1)
                at[side] = np.kron(Vs, kx(f))
            trs = {+1: ep, -1: em}
            for sk in (+1, -1):
                for sl in (+1, -1):
                    fac = [T0] * d
                    fac[dd] = np.einsum("a,b->ab", trs[sk], trs[sl])[:, :, None]
                    sp = fac[-1]
                    for F in reversed(fac[:-1]):
                        sp = _kron3(sp, F)
                    ga[(sk, sl)] = _kron3(T0, sp)       # (thT, thT, nPf)
            self.PsiAtFP.append(at)
            self.gamma.append(ga)


# ---------------------------------------------------------------------------
# residual, Jacobians, Newton
# ---------------------------------------------------------------------------
def _rusanov(flux, wL, wR, dd, alpha=None, pointwise=False):
    """Rusanov flux with alpha the largest wave speed on the face (one value per face, or
    one per face point if pointwise).  wL, wR: (m, E, q).  Returns (F-hat (m, E, q),
    alpha (E, 1) or (E, q)).  A given alpha is used as is (frozen)."""
    if alpha is None:
        alpha = np.maximum(flux.speed(wL, dd), flux.speed(wR, dd))
        if not pointwise:
            alpha = alpha.max(axis=-1, keepdims=True)
    Fh = 0.5 * (flux.F(wL, dd) + flux.F(wR, dd)) - 0.5 * alpha[None] * (wR - wL)
    return Fh, alpha


def _region_neighbours(d):
    offs = basis.region_offsets(d)
    index = {tuple(o): r for r, o in enumerate(offs)}
    nbrs = []
    for o in offs:
        row = {}
        for dd in range(d):
            for side in (+1, -1):
                o2 = o.copy()
                o2[dd] += side
                row[(dd, side)] = index.get(tuple(o2))
        nbrs.append(row)
    return offs, nbrs


def residual(W, Q, flux, tb: Tables, lam, frozen=None, pointwise=False):
    """R for a batch of regions.  W: (E, nR, m, thT), Q: (E, nR, m, thS).
    Returns (R, alpha) with alpha[(r, dd, side)] the face speeds ((E, 1), or (E, q) if
    pointwise).  With `frozen` (a previous alpha dict) the face speeds are not recomputed."""
    d = tb.d
    E, nR, m, _ = W.shape
    offs, nbrs = _region_neighbours(d)
    R = np.einsum("kl,erjl->erjk", tb.time_term, W)
    R -= np.einsum("ks,erjs->erjk", tb.source, Q)
    wv = np.einsum("erjk,kq->jerq", W, tb.PsiV)
    scale = [lam[dd] / 2.0 ** d for dd in range(d)]
    alphas = {}
    for dd in range(d):
        Fv = flux.F(wv, dd)
        R -= scale[dd] * np.einsum("kq,q,jerq->erjk", tb.dPsiV[dd], tb.wV, Fv)
        for r in range(nR):
            for side in (+1, -1):
                own = np.einsum("ejk,kq->jeq", W[:, r], tb.PsiF[dd][side])
                r2 = nbrs[r][(dd, side)]
                if r2 is None:
                    Fn = side * flux.F(own, dd)
                else:
                    nb_ = np.einsum("ejk,kq->jeq", W[:, r2], tb.PsiF[dd][-side])
                    fz = None if frozen is None else frozen[(r, dd, side)]
                    if side == +1:
                        Fh, al = _rusanov(flux, own, nb_, dd, fz, pointwise)
                    else:
                        Fh, al = _rusanov(flux, nb_, own, dd, fz, pointwise)
                    alphas[(r, dd, side)] = al
                    Fn = side * Fh
                R[:, r] += scale[dd] * np.einsum("kq,q,jeq->ejk", tb.PsiF[dd][side], tb.wF[dd], Fn)
    return R, alphas


def _project(Pbasis, wts, vals, norm):
    """Coefficients of vals (..., q) on an orthonormal (average-sense) basis."""
    return np.einsum("pq,q,...q->...p", Pbasis, wts, vals) / norm


def jacobian(W, Q, flux, tb: Tables, lam, alphas, kind: str = "qqf"):
    """Dense region Jacobian (E, n, n), n = nR m thT; kind 'qqf' or 'quad'."""
    d = tb.d
    E, nR, m, thT = W.shape
    offs, nbrs = _region_neighbours(d)
    J = np.zeros((E, nR, m, thT, nR, m, thT))
    scale = [lam[dd] / 2.0 ** d for dd in range(d)]
    for r in range(nR):
        for j in range(m):
            J[:, r, j, :, r, j, :] += tb.time_term
    eye = np.eye(m)[:, :, None, None]
    for dd in range(d):
        if kind == "qqf":
            wp = np.einsum("erjk,kq->jerq", W, tb.PsiAtP)
            Fp = _project(tb.PsiP, tb.wP, flux.dF(wp, dd), 2.0 ** (d + 1))  # (m,m,E,nR,nP)
            Jv = np.einsum("klp,ijerp->erikjl", tb.beta[dd], Fp)
        else:
            wv = np.einsum("erjk,kq->jerq", W, tb.PsiV)
            dF = flux.dF(wv, dd)
            Jv = np.einsum("kq,lq,q,ijerq->erikjl", tb.dPsiV[dd], tb.PsiV, tb.wV, dF)
        for r in range(nR):
            J[:, r, :, :, r, :, :] -= scale[dd] * Jv[:, r]
        for r in range(nR):
            for side in (+1, -1):
                r2 = nbrs[r][(dd, side)]
                if kind == "qqf":
                    at_own, at_nb = tb.PsiAtFP[dd][side], tb.PsiAtFP[dd][-side]
                    own = np.einsum("ejk,kq->jeq", W[:, r], at_own)
                else:
                    own = np.einsum("ejk,kq->jeq", W[:, r], tb.PsiF[dd][side])
                if r2 is None:
                    blocks = [(r, side, flux.dF(own, dd) * side)]
                else:
                    al = alphas[(r, dd, side)][None, None]
                    if kind == "qqf":
                        nbv = np.einsum("ejk,kq->jeq", W[:, r2], at_nb)
                    else:
                        nbv = np.einsum("ejk,kq->jeq", W[:, r2], tb.PsiF[dd][-side])
                    if al.shape[-1] != 1:
                        # pointwise speeds: this iterate's, at the points used here
                        al = np.maximum(flux.speed(own, dd), flux.speed(nbv, dd))[None, None]
                    # d F-hat / d w_L = (F'(w_L) + alpha I)/2, d/d w_R = (F'(w_R) - alpha I)/2
                    if side == +1:   # own is L, neighbour is R
                        g_own = 0.5 * (flux.dF(own, dd) + al * eye)
                        g_nb = 0.5 * (flux.dF(nbv, dd) - al * eye)
                    else:            # own is R, neighbour is L; F-hat . n = -F-hat
                        g_own = -0.5 * (flux.dF(own, dd) - al * eye)
                        g_nb = -0.5 * (flux.dF(nbv, dd) + al * eye)
                    blocks = [(r, side, g_own), (r2, -side, g_nb)]
                for (rl, sl, G) in blocks:
                    if kind == "qqf":
                        Gp = _project(tb.PsiFP[dd], tb.wFP[dd], G, 2.0 ** d)   # (m,m,E,nPf)
                        blk = np.einsum("klp,ijep->eikjl", tb.gamma[dd][(side, sl)], Gp)
                    else:
                        blk = np.einsum("kq,lq,q,ijeq->eikjl", tb.PsiF[dd][side],
                                        tb.PsiF[dd][sl], tb.wF[dd], G)
                    J[:, r, :, :, rl, :, :] += scale[dd] * blk
    n = nR * m * thT
    return J.reshape(E, n, n)


def newton_predict(Q, w, dt, kind="qqf", max_iters=4, tol=1e-10, chunk=16, cells=None,
                   return_iters=False, alpha="frozen"):
    """Centre-element W (cells, m*thT) for every cell (or the listed `cells`).
    alpha: "frozen" (Rusanov speeds of the initial iterate held fixed), "live" (per-face
    speeds of every iterate) or "point" (pointwise speeds of every iterate)."""
    if alpha not in ("frozen", "live", "point"):
        raise ValueError(alpha)
    pointwise = alpha == "point"
    d, M = w["dim"], w["M"]
    tb = Tables(d, M)
    flux = flux_model(w)
    m = flux.m
    lam = dt / cell_sizes(w)
    ncell = Q.shape[0]
    cells = np.arange(ncell) if cells is None else np.asarray(cells)
    Qr = Q.reshape(ncell, m, tb.thS)
    rc = (3 ** d - 1) // 2
    out = np.empty((len(cells), m * tb.thT))
    iters = np.zeros(len(cells), dtype=np.int64)
    conv = np.zeros(len(cells), dtype=bool)
    from .linear import gather_cells
    for c0 in range(0, len(cells), chunk):
        sel = cells[c0:c0 + chunk]
        QR = gather_cells(Q, w, sel).reshape(len(sel), 3 ** d, m, tb.thS)
        W = np.zeros((len(sel), 3 ** d, m, tb.thT))
        W[..., : tb.thS] = QR          # Q^n extended constant in time
        active = np.ones(len(sel), dtype=bool)
        it = np.zeros(len(sel), dtype=np.int64)
        # face speeds of the Rusanov flux, frozen at the initial iterate
        _, alpha0 = residual(W, QR, flux, tb, lam, pointwise=pointwise)
        for _ in range(max_iters):
            idx = np.nonzero(active)[0]
            if idx.size == 0:
                break
            al_idx = {k: v[idx] for k, v in alpha0.items()} if alpha == "frozen" else None
            R, al = residual(W[idx], QR[idx], flux, tb, lam, frozen=al_idx, pointwise=pointwise)
            J = jacobian(W[idx], QR[idx], flux, tb, lam, al, kind)
            delta = np.linalg.solve(J, R.reshape(idx.size, -1, 1)).reshape(R.shape)
            W[idx] -= delta
            it[idx] += 1
            dn = np.abs(delta).reshape(idx.size, -1).max(axis=1)
            wn = np.abs(W[idx]).reshape(idx.size, -1).max(axis=1)
            done = dn <= tol * np.maximum(1.0, wn)
            active[idx[done]] = False
        out[c0:c0 + len(sel)] = W[:, rc].reshape(len(sel), -1)
        iters[c0:c0 + len(sel)] = it
        conv[c0:c0 + len(sel)] = ~active
    if return_iters:
        return out, iters, conv
    return out


def correct(Q, Wc, w, dt, pointwise=False):
    """Q^{n+1} from Q^n and every cell's predicted W (cells, m*thT); the Rusanov speed per
    face (or per face point if pointwise) from the predicted traces."""
    d, M = w["dim"], w["M"]
    tb = Tables(d, M)
    flux = flux_model(w)
    m = flux.m
    lam = dt / cell_sizes(w)
    ncell = Q.shape[0]
    g = grid_shape(w)
    Wr = Wc.reshape(ncell, m, tb.thT)
    dQ = np.zeros((ncell, m, tb.thS))
    wv = np.einsum("ejk,kq->jeq", Wr, tb.PsiV)
    for dd in range(d):
        sc = lam[dd] / 2.0 ** d
        dQ += sc * np.einsum("sq,q,jeq->ejs", tb.dPhiV[dd], tb.wV, flux.F(wv, dd))
        own_p = np.einsum("ejk,kq->jeq", Wr, tb.PsiF[dd][+1])     # at xi_d = +1
        own_m = np.einsum("ejk,kq->jeq", Wr, tb.PsiF[dd][-1])     # at xi_d = -1
        ax = cell_axis(d, dd)
        right_m = np.roll(own_m.reshape((m,) + g + (-1,)), -1, axis=1 + ax).reshape(own_m.shape)
        Fh, _ = _rusanov(flux, own_p, right_m, dd, None, pointwise)  # face i+1/2, once
        dQ -= sc * np.einsum("sq,q,jeq->ejs", tb.PhiF[dd][+1], tb.wF[dd], Fh)
        Fl = np.roll(Fh.reshape((m,) + g + (-1,)), 1, axis=1 + ax).reshape(Fh.shape)
        dQ += sc * np.einsum("sq,q,jeq->ejs", tb.PhiF[dd][-1], tb.wF[dd], Fl)
    return Q + dQ.reshape(Q.shape)


def step(Q, w, dt, kind="qqf", max_iters=4, tol=1e-10, alpha="frozen"):
    W = newton_predict(Q, w, dt, kind=kind, max_iters=max_iters, tol=tol, alpha=alpha)
    return correct(Q, W, w, dt, pointwise=alpha == "point")


def max_speed(Q, w, npts: int = 6):
    """Largest wave speed of the state over a tensor grid of points in every cell."""
    d, M = w["dim"], w["M"]
    flux = flux_model(w)
    nb = M + 1
    x = np.linspace(-1.0, 1.0, npts)
    Phi = basis.kron_x_fastest([basis.phi(nb, x)] * d)
    vals = np.einsum("ejs,sq->jeq", Q.reshape(Q.shape[0], flux.m, -1), Phi)
    return float(max(flux.speed(vals, dd).max() for dd in range(d)))
