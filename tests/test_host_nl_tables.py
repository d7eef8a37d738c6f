"""Host-side (no GPU) checks of the nonlinear path's C++ tables and block elimination plan.

The library's host sources (nl_tables.cpp, tables.cpp) are compiled with g++ together with
tests/host/nl_host_check.cpp, which writes the tables the Newton kernel is given; they are
compared entry by entry with the oracle's Tables (basis values at the residual and
projection points, the projection factor, the triple-product integrals of eqs. Jacproj and
Jacobian2), and the merged per-(k, l) assembly lists are checked to contract to the same
region-cell blocks as the oracle's dense triple-product tensors.  The elimination plan
(corners, edges, centre, with its fill blocks) is checked against a dense LU solve.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import basis
from oracle import nonlinear as NL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_01231_gb300", "csrc")


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    return None


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("g++ or the CUDA runtime header is not available")
    out = str(tmp_path_factory.mktemp("nlhost") / "nl_host_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I" + inc, "-I" + CSRC,
                    os.path.join(ROOT, "tests", "host", "nl_host_check.cpp"),
                    os.path.join(CSRC, "nl_tables.cpp"), os.path.join(CSRC, "tables.cpp"),
                    "-o", out], check=True, capture_output=True)
    return out


def _tables(exe, M, tmp_path):
    path = str(tmp_path / f"t{M}.txt")
    subprocess.run([exe, "tables", str(M), path], check=True)
    out, lines, i = {}, open(path).read().split("\n"), 0
    while i < len(lines) and lines[i]:
        name, n = lines[i].split()
        n = int(n)
        out[name] = np.array([float(v) for v in lines[i + 1:i + 1 + n]])
        i += 1 + n
    return out


def _dense(ptr, p, val, npair, width):
    D = np.zeros((npair, width))
    for kl in range(npair):
        for e in range(int(ptr[kl]), int(ptr[kl + 1])):
            D[kl, int(p[e])] += val[e]
    return D


@pytest.mark.parametrize("M", [1, 2, 3])
def test_nl_tables_match_oracle(exe, M, tmp_path):
    c = _tables(exe, M, tmp_path)
    tb = NL.Tables(2, M)
    nb, thS, thT = M + 1, (M + 1) ** 2, (M + 1) ** 3
    npj = 2 * M + 1
    QP, QPf = npj ** 3, npj ** 2
    close = dict(rtol=1e-13, atol=1e-13)
    # time term psi_a(1) psi_g(1) - int psi_a' psi_g and the causal source psi_a(-1)
    np.testing.assert_allclose(c["Mt"].reshape(nb, nb), tb.time_term[::thS, ::thS], **close)
    np.testing.assert_allclose(c["em"], tb.source[::thS, 0], **close)
    # residual rule: volume and face values (tau slowest, then y, x)
    np.testing.assert_allclose(c["wV"], tb.wV, **close)
    np.testing.assert_allclose(c["PsiV"].reshape(thT, -1), tb.PsiV, **close)
    np.testing.assert_allclose(c["dPsiV"].reshape(2, thT, -1), np.stack(tb.dPsiV), **close)
    np.testing.assert_allclose(c["PhiV"].reshape(thS, -1), tb.PhiV, **close)
    np.testing.assert_allclose(c["dPhiV"].reshape(2, thS, -1), np.stack(tb.dPhiV), **close)
    Qf = tb.nq ** 2
    np.testing.assert_allclose(c["wF"].reshape(2, Qf), np.stack(tb.wF), **close)
    psf = c["PsiF"].reshape(2, 2, thT, Qf)
    phf = c["PhiF"].reshape(2, 2, thS, Qf)
    for dd in range(2):
        for si, side in enumerate((+1, -1)):
            np.testing.assert_allclose(psf[dd, si], tb.PsiF[dd][side], **close)
            np.testing.assert_allclose(phf[dd, si], tb.PhiF[dd][side], **close)
    # the 1D factors of the sum-factorised residual
    x, _ = basis.gauss(tb.nq)
    np.testing.assert_allclose(c["V1"].reshape(nb, -1), basis.phi(nb, x), **close)
    np.testing.assert_allclose(c["dV1"].reshape(nb, -1), basis.dphi(nb, x), **close)
    # projection rule: solution basis at the projection points, and the projection
    # (eq. Jacproj) as the tensor product of the 1D factor
    np.testing.assert_allclose(c["PsiAtP"].reshape(thT, QP), tb.PsiAtP, **close)
    pf = c["PsiAtFP"].reshape(2, 2, thT, QPf)
    for dd in range(2):
        for si, side in enumerate((+1, -1)):
            np.testing.assert_allclose(pf[dd, si], tb.PsiAtFP[dd][side], **close)
    P1 = c["P1"].reshape(npj, npj)
    np.testing.assert_allclose(np.kron(P1, np.kron(P1, P1)), tb.PsiP * tb.wP[None] / 8.0,
                               **close)
    # merged assembly lists: the diagonal block of a region cell takes the volume tensors
    # of both directions and the own-side face tensors of its four faces; the block towards
    # the neighbour across face f the neighbour-side tensor of that face
    # (the lists drop 1D factors below 1e-13: exact zeros the oracle's quadrature leaves
    # as rounding noise, up to ~1e-13 once multiplied by the other factors)
    lists = dict(rtol=1e-13, atol=1e-12)
    npair = thT * thT
    width = 2 * QP + 8 * QPf
    Dd = _dense(c["dptr"], c["doff"], c["dval"], npair, width)
    ref = np.zeros((npair, width))
    for dd in range(2):
        ref[:, dd * QP:(dd + 1) * QP] = tb.beta[dd].reshape(npair, QP)
    for f in range(4):
        dd, side = f >> 1, (+1, -1)[f & 1]
        o = 2 * QP + f * QPf
        ref[:, o:o + QPf] = tb.gamma[dd][(side, side)].reshape(npair, QPf)
    np.testing.assert_allclose(Dd, ref, **lists)
    for f in range(4):
        dd, side = f >> 1, (+1, -1)[f & 1]
        Do = _dense(c[f"optr{f}"], c[f"ooff{f}"], c[f"oval{f}"], npair, width)
        ref = np.zeros((npair, width))
        o = 2 * QP + (4 + f) * QPf
        ref[:, o:o + QPf] = tb.gamma[dd][(side, -side)].reshape(npair, QPf)
        np.testing.assert_allclose(Do, ref, **lists)


def test_elimination_plan_solves_region_system(exe):
    r = subprocess.run([exe, "plan"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "slots 43" in r.stdout        # 9 diagonal + 24 neighbour + 10 fill blocks
