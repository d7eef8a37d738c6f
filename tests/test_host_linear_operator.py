"""Host-side (no GPU) check of the linear path's centre-row operator.

The library's tables.cpp is compiled with g++ together with tests/host/lin_host_check.cpp,
which writes the operator P the prediction kernels are given: W_centre = P X over the
upwind box of region cells only.  It is compared with the oracle's dense solve of the
region system of eq. pred_full_system (all 3^d region cells): on the box's cells the
columns agree, and every region cell outside the box has a zero column -- with upwind
face values the centre depends only on the cells upstream of it.
"""
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import basis
from oracle import linear as OL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_01231_gb300", "csrc")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is not available")
    out = str(tmp_path_factory.mktemp("linhost") / "lin_host_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I" + CSRC,
                    os.path.join(ROOT, "tests", "host", "lin_host_check.cpp"),
                    os.path.join(CSRC, "tables.cpp"), "-o", out], check=True,
                   capture_output=True)
    return out


def _operator(exe, d, M, nu, tmp_path, fused=False):
    path = str(tmp_path / "P.txt")
    nu3 = list(nu) + [0.0] * (3 - len(nu))
    subprocess.run([exe, str(d), str(M)] + [repr(float(v)) for v in nu3] + [path]
                   + (["fused"] if fused else []), check=True, capture_output=True)
    lines = open(path).read().split()
    lo, cnt = [int(v) for v in lines[0:3]], [int(v) for v in lines[3:6]]
    n, size = int(lines[6]), int(lines[7])
    P = np.array([float(v) for v in lines[8:8 + size]])
    return lo, cnt, n, P


CASES = [
    (1, 3, (0.9,)), (1, 6, (-0.45,)), (1, 2, (0.0,)),
    (2, 1, (0.35, 0.175)), (2, 3, (0.35, 0.175)), (2, 2, (-0.3, 0.2)), (2, 3, (0.3, -0.7)),
    (2, 2, (0.0, -0.4)), (2, 4, (0.35, -0.35)), (2, 5, (-0.35, 0.2)),
    (3, 1, (0.3, 0.21, 0.09)), (3, 2, (0.3, -0.21, 0.0)),
    (3, 1, (-0.6, -0.6, 0.6)), (3, 3, (0.3, -0.21, 0.09)),
]


@pytest.mark.parametrize("d,M,nu", CASES)
def test_upwind_operator_matches_oracle_region_solve(exe, d, M, nu, tmp_path):
    lo, cnt, n, P = _operator(exe, d, M, nu, tmp_path)
    nb = M + 1
    thS, thT = nb ** d, nb ** (d + 1)
    # the box: {-1, 0} upstream of a positive velocity, {0, +1} of a negative, {0} if zero
    for dd in range(3):
        v = nu[dd] if dd < d else 0.0
        assert (lo[dd], cnt[dd]) == ((-1, 2) if v > 0 else (0, 2) if v < 0 else (0, 1))
    assert n == cnt[0] * cnt[1] * cnt[2]
    P = P.reshape(thT, n * thS)
    A, B = OL.region_system(d, M, np.asarray(nu))
    rc = (3 ** d - 1) // 2
    G = sla.solve(A, B)[rc * thT:(rc + 1) * thT]        # (theta_T, 3^d theta_S)
    scale = np.abs(G).max()
    offs = [tuple(o) for o in basis.region_offsets(d)]
    box = list(itertools.product(*[range(lo[dd], lo[dd] + cnt[dd]) for dd in range(d)][::-1]))
    box = [tuple(reversed(o)) for o in box]              # x fastest
    seen = set()
    for i, o in enumerate(box):
        r = offs.index(o)
        seen.add(r)
        np.testing.assert_allclose(P[:, i * thS:(i + 1) * thS], G[:, r * thS:(r + 1) * thS],
                                   rtol=0, atol=1e-12 * scale)
    for r in range(len(offs)):
        if r not in seen:
            assert np.abs(G[:, r * thS:(r + 1) * thS]).max() <= 1e-13 * scale


def _step_symbol(d, M, nu, P, lo, cnt, theta):
    """Amplification matrix of one linear RIDG step (prediction with the host operator P over
    the upwind box, then the correction of Sec. 2.3) for the Fourier mode e^{i theta . j}."""
    nb = M + 1
    thS = nb ** d
    D = basis.deriv_matrix(nb)
    ep, em = basis.trace_plus(nb), basis.trace_minus(nb)

    def along(dd, X):
        mats = [np.eye(nb)] * d
        mats[dd] = X
        return basis.kron_x_fastest(mats)

    n = cnt[0] * cnt[1] * cnt[2]
    Wb = np.zeros((thS, thS), dtype=complex)
    for i in range(n):
        o = (lo[0] + i % cnt[0], lo[1] + (i // cnt[0]) % cnt[1], lo[2] + i // (cnt[0] * cnt[1]))
        Wb += P[:thS, i * thS:(i + 1) * thS] * np.exp(1j * sum(theta[k] * o[k] for k in range(d)))
    G = np.eye(thS, dtype=complex)
    for dd in range(d):
        ph = np.exp(1j * theta[dd])
        nup, num = max(nu[dd], 0.0), min(nu[dd], 0.0)
        # face value at +1/2: nu+ tr+(W_i) + nu- tr-(W_{i+e}), distributed with phi(+1); at
        # -1/2 the same value shifted by -e, distributed with phi(-1)
        Fp = along(dd, np.outer(ep, ep) * nup + np.outer(ep, em) * num * ph)
        Fm = along(dd, (np.outer(em, ep) * nup + np.outer(em, em) * num * ph) / ph)
        G = G + (nu[dd] * along(dd, D) - Fp + Fm) @ Wb
    return G


def test_step_symbol_matches_oracle_step(exe, tmp_path):
    # the symbol built from the host operator equals the oracle's own step on a Fourier mode
    d, M, N = 3, 1, 4
    vel = (1.0, -0.7, 0.4)
    w = dict(flux="advection", dim=d, n=(N,) * d, M=M, vel=vel, lo=(0.0,) * d, hi=(1.0,) * d)
    dt = 0.6 / N
    nu = np.asarray(vel) * dt * N
    lo, cnt, n, P = _operator(exe, d, M, nu, tmp_path)
    nb = M + 1
    thS, thT = nb ** d, nb ** (d + 1)
    P = P.reshape(thT, n * thS)
    j = np.stack(np.meshgrid(*[np.arange(N)] * d, indexing="ij"), -1).reshape(-1, d)[:, ::-1]
    for k in ((1, 2, 3), (0, 1, 0), (3, 3, 1)):
        theta = 2 * np.pi * np.asarray(k) / N
        phase = np.exp(1j * (j @ theta))
        Go = np.zeros((thS, thS), dtype=complex)
        for s in range(thS):
            e = np.zeros(thS)
            e[s] = 1.0
            out = OL.step(np.real(phase)[:, None] * e, w, dt) + \
                1j * OL.step(np.imag(phase)[:, None] * e, w, dt)
            Go[:, s] = out[0]                # cell 0 carries the mode's amplitude
        np.testing.assert_allclose(_step_symbol(d, M, nu, P, lo, cnt, theta), Go, atol=1e-13)


def test_3d_cfl_readings(exe, tmp_path):
    # The paper's 3D runs use nu = 0.6 with a = (1, 1, 1).  Per direction (dt = nu h / max
    # |a_d|) the step grows at degree 3 (spectral radius 1.04 on this 8^3 wavenumber grid,
    # 1.048 on a 12^3 one: a few percent per step); as dt = nu h / sum_d |a_d| (0.2 per
    # direction) it is stable.
    d, M = 3, 3
    grid = 2 * np.pi * np.arange(8) / 8
    rho = {}
    for nud in (0.6, 0.2):
        nu = np.full(3, nud)
        lo, cnt, n, P = _operator(exe, d, M, nu, tmp_path)
        P = P.reshape((M + 1) ** 4, n * (M + 1) ** 3)
        rho[nud] = max(np.abs(np.linalg.eigvals(_step_symbol(d, M, nu, P, lo, cnt, th))).max()
                       for th in itertools.product(grid, repeat=3))
    assert rho[0.6] > 1.03, rho
    assert rho[0.2] <= 1.0 + 1e-10, rho


FUSED_CASES = [
    (2, 3, (0.35, 0.175)), (2, 2, (-0.3, 0.2)), (2, 1, (0.0, -0.4)),
    (3, 2, (0.3, -0.21, 0.09)), (3, 1, (-0.2, 0.0, 0.25)), (3, 2, (0.0, 0.3, -0.2)),
]


@pytest.mark.parametrize("d,M,nu", FUSED_CASES)
def test_fused_step_operator_reproduces_oracle_step(exe, d, M, nu, tmp_path):
    """The mixed path's fused step operator (host-built G = C P-bar: the volume term and,
    per direction and line of modes, the cell's upwind trace on its downstream face), applied
    to every cell's upwind box and assembled into the update the way the correction kernels
    do it -- F(i - 1/2) the upstream cell's trace output, F(i + 1/2) this cell's (the other
    way round for a negative velocity), mode a of a line getting phi_a(+1) ((-1)^a F(i - 1/2)
    - F(i + 1/2)) -- gives the oracle's step (its region solves and correction)."""
    lo, cnt, n, G = _operator(exe, d, M, nu, tmp_path, fused=True)
    nb = M + 1
    thS, NT = nb ** d, nb ** (d - 1)
    G = G.reshape(thS + d * NT, n * thS)
    mesh = (5, 4) if d == 2 else (4, 3, 3)
    n3 = list(mesh) + [1] * (3 - d)
    vel = [nu[k] / mesh[k] for k in range(d)] + [0.0] * (3 - d)   # nu = vel dt / h at dt = 1
    w = dict(flux="advection", dim=d, n=mesh, M=M, vel=tuple(vel), lo=(0.0,) * 3,
             hi=(1.0,) * 3)
    cells = int(np.prod(mesh))
    Q = np.random.default_rng(5).standard_normal((cells, thS))

    def cell(x, y, z):
        return (x % n3[0]) + n3[0] * ((y % n3[1]) + n3[1] * (z % n3[2]))

    box = [(lo[0] + i % cnt[0], lo[1] + (i // cnt[0]) % cnt[1], lo[2] + i // (cnt[0] * cnt[1]))
           for i in range(n)]
    Y = np.zeros((cells, G.shape[0]))
    for z in range(n3[2]):
        for y in range(n3[1]):
            for x in range(n3[0]):
                X = np.concatenate([Q[cell(x + o[0], y + o[1], z + o[2])] for o in box])
                Y[cell(x, y, z)] = G @ X
    ep = basis.trace_plus(nb)
    out = Q.copy()
    for z in range(n3[2]):
        for y in range(n3[1]):
            for x in range(n3[0]):
                e = cell(x, y, z)
                dq = Y[e, :thS].copy()
                for dd in range(d):
                    if nu[dd] == 0.0:
                        continue
                    step = [0, 0, 0]
                    step[dd] = -1 if nu[dd] > 0 else 1
                    up = cell(x + step[0], y + step[1], z + step[2])
                    st = nb ** dd
                    for t in range(NT):
                        base = (t % st) + (t // st) * st * nb
                        fo = Y[e, thS + dd * NT + t]
                        fu = Y[up, thS + dd * NT + t]
                        fm, fp = (fu, fo) if nu[dd] > 0 else (fo, fu)
                        for a in range(nb):
                            dq[base + a * st] += ep[a] * ((-1) ** a * fm - fp)
                out[e] += dq
    ref = OL.step(Q, w, 1.0)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
