"""Seeded synthetic inputs for the RIDG workloads.

This module produces initial data and exact solutions as cell-wise coefficients in
the orthonormal tensor Legendre basis of Sec. 2.1 (Phi_s = prod_d sqrt(2 b_d + 1) P_{b_d},
normalised so that (1/|T|) int_T Phi_k Phi_l = delta_kl), ordered x-fastest.  It holds
none of the prediction / correction arithmetic: both the CUDA path and the oracle take
their inputs from here, so that neither depends on the other.

Workload parameters (mesh, degree, velocity, CFL number, final time) are the synthetic
stand-ins for the paper's analytic test problems (eqs. adv1d, adv2d, burger2d, adv3d);
the sine / Fourier / vortex initial data replace the paper's bump profiles.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg

# ---------------------------------------------------------------------------
# workload table
# ---------------------------------------------------------------------------
WORKLOADS = {
    # 1D advection u_t + u_x = 0 on [0,1], 64 cells, degree 3, u0 = sin(2 pi x)
    "adv1d_n64_q3": dict(flux="advection", dim=1, n=(64,), M=3, vel=(1.0,),
                         lo=(0.0,), hi=(1.0,), cfl=0.45, T=1.0, ic="sin"),
    # 2D advection u_t + u_x + 0.5 u_y = 0 on [0,1]^2, 256^2 cells, Q3
    "adv2d_n256_q3": dict(flux="advection", dim=2, n=(256, 256), M=3, vel=(1.0, 0.5),
                          lo=(0.0, 0.0), hi=(1.0, 1.0), cfl=0.35, T=1.0, ic="sin"),
    # 3D advection with velocity (1, 0.7, 0.3) on [0,1]^3, 96^3 cells, Q2,
    # product of sines plus seeded uniform 1e-3 coefficient noise
    "adv3d_n96_q2": dict(flux="advection", dim=3, n=(96, 96, 96), M=2,
                         vel=(1.0, 0.7, 0.3), lo=(0.0,) * 3, hi=(1.0,) * 3,
                         cfl=0.30, T=1.0, ic="sin+noise"),
    # the paper's 2D and 3D advection studies (eqs. adv2d, adv3d): the C-infinity bump
    # (paper_bump), a = (1, ..., 1), degree 5, its nu = 0.7 (2D) / 0.6 (3D) taken as
    # dt = nu h / sum_d |a_d|
    "adv2d_bump_n60_q5": dict(flux="advection", dim=2, n=(60, 60), M=5, vel=(1.0, 1.0),
                              lo=(0.0, 0.0), hi=(1.0, 1.0), cfl=0.35, T=1.0, ic="bump"),
    "adv3d_bump_n48_q5": dict(flux="advection", dim=3, n=(48, 48, 48), M=5,
                              vel=(1.0, 1.0, 1.0), lo=(0.0,) * 3, hi=(1.0,) * 3, cfl=0.2,
                              T=1.0, ic="bump"),
    # 2D compressible Euler, isentropic vortex on [0,10]^2, 512^2 cells, Q2
    "euler2d_n512_q2": dict(flux="euler", dim=2, n=(512, 512), M=2, gamma=1.4,
                            lo=(0.0, 0.0), hi=(10.0, 10.0), cfl=0.35, T=1.0,
                            ic="vortex"),
}


def workload(name: str, **override) -> dict:
    """Parameters of a named workload; keyword overrides (e.g. a smaller mesh)."""
    w = dict(WORKLOADS[name])
    w.update(override)
    w["name"] = name
    return w


# ---------------------------------------------------------------------------
# 1D Legendre helpers (library evaluation of P_b; used only to project data)
# ---------------------------------------------------------------------------
def _legendre_orthonormal(nb: int, x: np.ndarray) -> np.ndarray:
    """V[b, ...] = sqrt(2b+1) P_b(x)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((nb,) + x.shape)
    for b in range(nb):
        c = np.zeros(b + 1)
        c[b] = 1.0
        out[b] = math.sqrt(2 * b + 1) * npleg.legval(x, c)
    return out


def _cell_points(n: int, lo: float, hi: float, nq: int):
    """Gauss points of every cell: x[i, q], reference weights w[q] (sum 2), V[b, q]."""
    xi, w = npleg.leggauss(nq)
    h = (hi - lo) / n
    centres = lo + (np.arange(n) + 0.5) * h
    return centres[:, None] + 0.5 * h * xi[None, :], w, xi


def project_1d(f, n: int, lo: float, hi: float, nb: int, nq: int | None = None) -> np.ndarray:
    """c[i, b] = (1/h) int_{cell i} f(x) phi_b(x) dx for a 1D function f."""
    nq = nq or nb + 8
    x, w, xi = _cell_points(n, lo, hi, nq)
    V = _legendre_orthonormal(nb, xi)
    return 0.5 * np.einsum("iq,q,bq->ib", f(x), w, V)


def _outer_modes(factors):
    """Combine per-dimension coefficient tables c_d[i_d, b_d] (d = 0 is x) into
    c[cells (z, y, x) ..., modes x-fastest]."""
    d = len(factors)
    out = factors[0]  # (nx, nb)
    for k in range(1, d):
        f = factors[k]
        # out: (cells_prev..., modes_prev) ; f: (n_k, nb)
        out = np.einsum("...m,ib->i...bm", out, f)
        # merge mode axes: new modes index = b * prev + m  (x fastest)
        sh = out.shape
        out = out.reshape(sh[:-2] + (sh[-2] * sh[-1],))
    return out


def project_separable(fs, w: dict, nb: int, nq: int | None = None) -> np.ndarray:
    """Coefficients of prod_d fs[d](x_d) on the workload's mesh, shape (cells, nb^d)."""
    d = w["dim"]
    facs = [project_1d(fs[k], w["n"][k], w["lo"][k], w["hi"][k], nb, nq) for k in range(d)]
    c = _outer_modes(facs)
    return c.reshape(-1, nb ** d)


def project_tensor(f, w: dict, nb: int, nq: int | None = None, m: int = 1,
                   chunk: int = 64) -> np.ndarray:
    """Coefficients of a general f(x, y[, z]) -> (m, ...) by tensor Gauss quadrature.
    Returns shape (cells, m, nb^d).  Cells are processed in slabs of the slowest axis."""
    d = w["dim"]
    nq = nq or nb + 8
    xi, wq = npleg.leggauss(nq)
    V = _legendre_orthonormal(nb, xi)  # (nb, nq)
    n = w["n"]
    h = [(w["hi"][k] - w["lo"][k]) / n[k] for k in range(d)]
    pts = [w["lo"][k] + (np.arange(n[k]) + 0.5)[:, None] * h[k] + 0.5 * h[k] * xi[None, :]
           for k in range(d)]  # pts[k][i, q]
    ncell = int(np.prod(n))
    out = np.empty((ncell, m, nb ** d))
    if d == 1:
        vals = np.asarray(f(pts[0])).reshape(m, n[0], nq)
        c = 0.5 * np.einsum("rip,p,bp->irb", vals, wq, V)
        out[:] = c
        return out
    if d == 2:
        X = pts[0][None, :, None, :]   # (1, nx, 1, qx)
        for j0 in range(0, n[1], chunk):
            j1 = min(n[1], j0 + chunk)
            Y = pts[1][j0:j1, None, :, None]  # (ny', 1, qy, 1)
            Xb, Yb = np.broadcast_arrays(X, Y)
            vals = np.asarray(f(Xb, Yb)).reshape(m, j1 - j0, n[0], nq, nq)
            # modes: s = bx + nb * by
            c = 0.25 * np.einsum("rjipq,p,q,cp,bq->jircb", vals, wq, wq, V, V)
            out[j0 * n[0]:j1 * n[0]] = c.reshape((j1 - j0) * n[0], m, nb * nb)
        return out
    X = pts[0][None, None, :, None, None, :]
    Y = pts[1][None, :, None, None, :, None]
    for k0 in range(0, n[2], max(1, chunk // 8)):
        k1 = min(n[2], k0 + max(1, chunk // 8))
        Z = pts[2][k0:k1, None, None, :, None, None]
        Xb, Yb, Zb = np.broadcast_arrays(X, Y, Z)
        vals = np.asarray(f(Xb, Yb, Zb)).reshape(m, k1 - k0, n[1], n[0], nq, nq, nq)
        c = 0.125 * np.einsum("rkjiopq,o,p,q,ao,bp,cq->kjirabc", vals, wq, wq, wq, V, V, V)
        out[k0 * n[0] * n[1]:k1 * n[0] * n[1]] = c.reshape(-1, m, nb ** 3)
    return out


def paper_bump(*xs, c: float = 0.5, omega: float = 1.0 / 3.0):
    """The C-infinity bump of the paper's advection studies (eqs. adv1d, adv2d, adv3d):
    exp(1 / (|x - c|^2 - omega^2)) inside the ball |x - c| < omega, 0 outside."""
    r2 = sum((np.asarray(x) - c) ** 2 for x in xs)
    out = np.zeros(np.broadcast(*xs).shape)
    m = r2 < omega * omega
    out[m] = np.exp(1.0 / (r2[m] - omega * omega))
    return out


def project_bump(w: dict, nb: int, nq: int = 20, c: float = 0.5,
                 omega: float = 1.0 / 3.0) -> np.ndarray:
    """L2 projection of paper_bump onto the orthonormal tensor basis of w's mesh (dim 1-3),
    shape (cells, nb^d), by tensor Gauss quadrature with nq points per dimension summed one
    dimension at a time; cells that do not meet the bump's ball stay zero."""
    d = w["dim"]
    n = list(w["n"])
    xi, wq = npleg.leggauss(nq)
    Vw = _legendre_orthonormal(nb, xi) * wq[None, :]      # (nb, nq)
    h = [(w["hi"][k] - w["lo"][k]) / n[k] for k in range(d)]
    lo = [w["lo"][k] for k in range(d)]
    pts = [lo[k] + (np.arange(n[k]) + 0.5)[:, None] * h[k] + 0.5 * h[k] * xi[None, :]
           for k in range(d)]                             # pts[k][i, q]
    # squared distance from c to the nearest point of each cell, per axis
    near = [np.maximum(0.0, np.abs(lo[k] + (np.arange(n[k]) + 0.5) * h[k] - c) - 0.5 * h[k]) ** 2
            for k in range(d)]
    out = np.zeros((int(np.prod(n)), nb ** d))
    if d == 1:
        vals = paper_bump(pts[0], c=c, omega=omega)      # (i, q)
        out[:] = 0.5 * vals @ Vw.T
        return out
    if d == 2:
        for j in range(n[1]):
            if near[1][j] >= omega * omega:
                continue
            X = pts[0][:, None, :]                        # (i, 1, qx)
            Y = pts[1][j][None, :, None]                  # (1, qy, 1)
            vals = paper_bump(X, Y, c=c, omega=omega)     # (i, p, q)
            t = np.tensordot(vals, Vw, axes=([2], [1]))   # (i, p, bx)
            t = np.tensordot(t, Vw, axes=([1], [1]))      # (i, bx, by)
            out[j * n[0]:(j + 1) * n[0]] = 0.25 * t.transpose(0, 2, 1).reshape(n[0], nb * nb)
        return out
    for k in range(n[2]):
        if near[2][k] >= omega * omega:
            continue
        js = [j for j in range(n[1]) if near[2][k] + near[1][j] < omega * omega]
        if not js:
            continue
        X = pts[0][None, :, None, None, :]                # (1, i, 1, 1, qx)
        Y = pts[1][js][:, None, None, :, None]            # (j, 1, 1, qy, 1)
        Z = pts[2][k][None, None, :, None, None]          # (1, 1, qz, 1, 1)
        vals = paper_bump(X, Y, Z, c=c, omega=omega)      # (j, i, o, p, q)
        t = np.tensordot(vals, Vw, axes=([4], [1]))       # (j, i, o, p, bx)
        t = np.tensordot(t, Vw, axes=([3], [1]))          # (j, i, o, bx, by)
        t = np.tensordot(t, Vw, axes=([2], [1]))          # (j, i, bx, by, bz)
        t = 0.125 * t.transpose(0, 1, 4, 3, 2).reshape(len(js), n[0], nb ** 3)
        for jj, j in enumerate(js):
            e0 = (k * n[1] + j) * n[0]
            out[e0:e0 + n[0]] = t[jj]
    return out


# ---------------------------------------------------------------------------
# initial data and exact solutions
# ---------------------------------------------------------------------------
def _sin2pi(shift: float):
    return lambda x: np.sin(2.0 * np.pi * (x - shift))


def advection_noise(w: dict, seed: int = 0) -> np.ndarray:
    """i.i.d. U(-1e-3, 1e-3) added to every Q(M) coefficient of every cell (PCG64)."""
    nb = w["M"] + 1
    ncell = int(np.prod(w["n"]))
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1e-3, 1e-3, size=(ncell, nb ** w["dim"]))


def initial_state(w: dict, seed: int = 0) -> np.ndarray:
    """Initial coefficients Q^0 in the canonical layout, shape (cells, m * theta_S)."""
    nb = w["M"] + 1
    if w["flux"] == "advection" and w["ic"] == "bump":
        return np.ascontiguousarray(project_bump(w, nb, nq=16))
    if w["flux"] == "advection":
        q = project_separable([_sin2pi(0.0)] * w["dim"], w, nb)
        if w["ic"] == "sin+noise":
            q = q + advection_noise(w, seed)
        return np.ascontiguousarray(q)
    if w["flux"] == "euler":
        return np.ascontiguousarray(
            project_tensor(lambda x, y: vortex_state(x, y, 0.0, w.get("gamma", 1.4)), w, nb, m=4
                           ).reshape(-1, 4 * nb ** 2))
    if w["flux"] == "burgers":
        return np.ascontiguousarray(burgers_initial(w, nb))
    raise ValueError(w["flux"])


def exact_coefficients(w: dict, t: float, nb: int | None = None) -> np.ndarray:
    """Projection of the exact solution at time t onto Q(nb-1) cell-wise (default
    nb = M + 2, the Q(M+1) space the L2 error definition of Sec. 4 needs)."""
    nb = nb or w["M"] + 2
    if w["flux"] == "advection" and w["ic"] == "bump":
        # the bump carried by a t around the periodic unit domain: offered where a t is a
        # whole number of periods, i.e. the bump is back at its start
        shift = np.asarray(w["vel"][: w["dim"]], dtype=float) * t
        if np.abs(shift - np.round(shift)).max() > 1e-12:
            raise ValueError("bump: exact coefficients only where a t is a whole period")
        return np.ascontiguousarray(project_bump(w, nb, nq=16))
    if w["flux"] == "advection":
        if w["ic"] != "sin":
            raise ValueError("exact coefficients are available for the noise-free data only")
        a = w["vel"]
        return np.ascontiguousarray(
            project_separable([_sin2pi(a[k] * t) for k in range(w["dim"])], w, nb))
    if w["flux"] == "euler":
        return np.ascontiguousarray(
            project_tensor(lambda x, y: vortex_state(x, y, t, w.get("gamma", 1.4)), w, nb, m=4
                           ).reshape(-1, 4 * nb ** 2))
    if w["flux"] == "burgers":
        return np.ascontiguousarray(
            project_tensor(lambda x, y: burgers_exact(w, x, y, t), w, nb).reshape(-1, nb ** 2))
    raise ValueError(w["flux"])


# --- exact error of a translated piecewise polynomial (the noisy 3D data) -------
def shifted_polynomial_error(w: dict, Q0: np.ndarray, Q: np.ndarray, t: float) -> float:
    """Relative L2 error ||Q_h - q(., t)|| / ||q(., t)|| of coefficients Q (cells, theta_S)
    against the exact solution of linear advection from the piecewise polynomial Q0 (the
    same layout): q(x, t) = q0(x - a t), periodic.  Both are polynomials on each of the 2^d
    sub-boxes in which the shifted mesh cuts a cell, so the integral is exact with M + 2
    Gauss points per dimension on each sub-box; the denominator is ||q0||^2 = sum |T| Q0^2
    (orthonormal basis, translation preserves the integral)."""
    d, nb = w["dim"], w["M"] + 1
    n = tuple(int(v) for v in w["n"][:d])
    h = [(w["hi"][k] - w["lo"][k]) / n[k] for k in range(d)]
    shape = tuple(reversed(n)) + (nb,) * d          # (z, y, x, bz, by, bx)
    A = np.asarray(Q, dtype=np.float64).reshape(shape)
    B = np.asarray(Q0, dtype=np.float64).reshape(shape)
    ng = nb + 1
    xg, wg = npleg.leggauss(ng)
    # per dimension (x first): the sub-intervals of a cell, each with its points in the cell's
    # own coordinate, the matching points of the source cell and the source cell's offset
    subs = []
    for k in range(d):
        sh = w["vel"][k] * t / h[k]                 # shift in cells
        kk = math.floor(sh)
        f = sh - kk
        parts = []
        # xi in [-1, -1 + 2f]: source cell i - kk - 1 at xi + 2 - 2f
        # xi in [-1 + 2f, 1]: source cell i - kk at xi - 2f
        for lo_, hi_, off, dxi in ((-1.0, -1.0 + 2 * f, kk + 1, 2.0 - 2 * f),
                                   (-1.0 + 2 * f, 1.0, kk, -2 * f)):
            if hi_ - lo_ <= 0.0:
                continue
            xi = 0.5 * (hi_ - lo_) * xg + 0.5 * (hi_ + lo_)
            wt = 0.5 * (hi_ - lo_) * wg
            parts.append((_legendre_orthonormal(nb, xi), _legendre_orthonormal(nb, xi + dxi),
                          wt, off))
        subs.append(parts)
    axes = "zyx"[3 - d:]          # cell axes of A, slowest first
    modes = "cba"[3 - d:]         # mode axes: bz, by, bx
    pts = "rqp"[3 - d:]           # point axes
    num = 0.0
    import itertools
    for combo in itertools.product(*[range(len(subs[k])) for k in range(d)]):
        own, src = A, B
        src_shift = []
        for k in range(d):
            Vo, Vs, wt, off = subs[k][combo[k]]
            src_shift.append(off)
        # source cell i - off along each dimension: roll by +off
        src = np.roll(B, shift=[src_shift[k] for k in reversed(range(d))], axis=tuple(range(d)))
        vo, vs = own, src
        for k in range(d):               # contract the mode of dimension k (x = last)
            Vo, Vs, wt, off = subs[k][combo[k]]
            ax = d + (d - 1 - k)         # mode axis of dimension k in the current array
            vo = np.moveaxis(np.tensordot(vo, Vo, axes=([ax], [0])), -1, ax)
            vs = np.moveaxis(np.tensordot(vs, Vs, axes=([ax], [0])), -1, ax)
        diff2 = (vo - vs) ** 2
        wts = np.ones(())
        for k in reversed(range(d)):     # weights in axis order (z, y, x)
            wts = np.multiply.outer(wts, subs[k][combo[k]][2])
        num += float(np.tensordot(diff2, wts, axes=(list(range(d, 2 * d)), list(range(d)))).sum())
    vol_ref = 2.0 ** d                   # sum of the reference weights over a whole cell
    den = float((B ** 2).sum()) * vol_ref
    return math.sqrt(num / den)


# --- isentropic vortex (ambient (rho,u,v,p) = (1,1,1,1), strength 5, centre (5,5)) --
def vortex_state(x, y, t, gamma=1.4, eps=5.0, xc=5.0, yc=5.0, L=10.0):
    """Conserved variables (rho, rho u, rho v, E) of the translating isentropic vortex."""
    dx = x - (xc + t)
    dy = y - (yc + t)
    dx = dx - L * np.round(dx / L)
    dy = dy - L * np.round(dy / L)
    r2 = dx * dx + dy * dy
    f = np.exp(0.5 * (1.0 - r2))
    u = 1.0 - eps / (2 * np.pi) * f * dy
    v = 1.0 + eps / (2 * np.pi) * f * dx
    T = 1.0 - (gamma - 1.0) * eps ** 2 / (8 * gamma * np.pi ** 2) * f * f
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E])


# --- Burgers ensemble: 5 Fourier modes, amplitudes summing to 0.5 ---------------
def burgers_modes(seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = [(k, l) for k in range(-3, 4) for l in range(-3, 4) if (k, l) != (0, 0)]
    idx = rng.choice(len(ks), size=5, replace=False)
    kl = np.array([ks[i] for i in idx], dtype=np.float64)
    ph = rng.uniform(0.0, 2 * np.pi, size=5)
    a = rng.uniform(0.0, 1.0, size=5)
    a = 0.5 * a / a.sum()
    return kl, ph, a


def burgers_u0(modes, x, y):
    kl, ph, a = modes
    u = np.zeros(np.broadcast(x, y).shape)
    for m in range(len(a)):
        u = u + a[m] * np.cos(2 * np.pi * (kl[m, 0] * x + kl[m, 1] * y) + ph[m])
    return u


def burgers_u0_grad_sum(modes, x, y):
    kl, ph, a = modes
    g = np.zeros(np.broadcast(x, y).shape)
    for m in range(len(a)):
        g = g - a[m] * 2 * np.pi * (kl[m, 0] + kl[m, 1]) * np.sin(
            2 * np.pi * (kl[m, 0] * x + kl[m, 1] * y) + ph[m])
    return g


def burgers_ensemble(count: int = 64, seed: int = 0, nmin: int = 64, nmax: int = 512,
                     mmin: int = 1, mmax: int = 4, cfl: float = 0.35):
    """The batched ensemble: instance sizes N ~ U{nmin..nmax} (N x N), degrees
    M ~ U{mmin..mmax}, Fourier data seeded per instance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ns = rng.integers(nmin, nmax + 1, size=count)
    Ms = rng.integers(mmin, mmax + 1, size=count)
    out = []
    for i in range(count):
        out.append(dict(flux="burgers", dim=2, n=(int(Ns[i]), int(Ns[i])), M=int(Ms[i]),
                        lo=(0.0, 0.0), hi=(1.0, 1.0), cfl=cfl, T=None, ic="fourier",
                        seed=int(seed * 1000 + i), name=f"burgers_{i}"))
    return out


def burgers_initial(w: dict, nb: int) -> np.ndarray:
    modes = burgers_modes(w["seed"])
    kl, ph, a = modes
    facs = []
    # cos(2pi(kx+ly)+ph) = cos(2pi kx + ph) cos(2pi ly) - sin(2pi kx + ph) sin(2pi ly)
    c = 0.0
    for m in range(5):
        k, l = kl[m]
        cx = project_1d(lambda x: np.cos(2 * np.pi * k * x + ph[m]), w["n"][0], 0.0, 1.0, nb)
        sx = project_1d(lambda x: np.sin(2 * np.pi * k * x + ph[m]), w["n"][0], 0.0, 1.0, nb)
        cy = project_1d(lambda y: np.cos(2 * np.pi * l * y), w["n"][1], 0.0, 1.0, nb)
        sy = project_1d(lambda y: np.sin(2 * np.pi * l * y), w["n"][1], 0.0, 1.0, nb)
        c = c + a[m] * (_outer_modes([cx, cy]) - _outer_modes([sx, sy]))
    return c.reshape(-1, nb * nb)


def burgers_shock_time(w: dict) -> float:
    """t* = 1 / max(-(d/dx + d/dy) u0) for u_t + (u^2/2)_x + (u^2/2)_y = 0."""
    modes = burgers_modes(w["seed"])
    g = np.linspace(0, 1, 1025)
    X, Y = np.meshgrid(g, g, indexing="ij")
    m = np.max(-burgers_u0_grad_sum(modes, X, Y))
    return 1.0 / m


def burgers_exact(w: dict, x, y, t, iters: int = 60):
    """Pre-shock solution u = u0(x - u t, y - u t), solved pointwise by Newton."""
    modes = burgers_modes(w["seed"])
    u = burgers_u0(modes, x, y)
    for _ in range(iters):
        xs, ys = x - u * t, y - u * t
        g = u - burgers_u0(modes, xs, ys)
        dg = 1.0 + t * burgers_u0_grad_sum(modes, xs, ys)
        u = u - g / dg
    return u
