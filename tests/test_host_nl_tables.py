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


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_factorised_assembly_matches_oracle_tensors(exe, M, tmp_path):
    """The FP32 Newton kernels assemble a region cell's blocks (one conserved variable) by
    sum factorisation: the projected arrays are contracted with the 1D triple products one
    dimension at a time (x, then y, then time), the face terms folded in with their trace
    pairs.  The same contractions written out here with the host's 1D factors, in the
    kernel's index conventions, give the blocks the oracle's dense triple-product tensors
    give (eqs. Jacproj, Jacobian2): the diagonal block (volume of both directions, own sides
    of the four faces) and the block towards the neighbour across each face."""
    c = _tables(exe, M, tmp_path)
    tb = NL.Tables(2, M)
    nb, npj = M + 1, 2 * M + 1
    thT, QP, QPf = nb ** 3, npj ** 3, npj ** 2
    T0 = c["T0"].reshape(nb, nb, npj)
    T1 = c["T1"].reshape(nb, nb, npj)
    ep, em = c["ep1"], c["em1"]
    np.testing.assert_allclose(ep, basis.phi(nb, np.array([1.0]))[:, 0], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(em, basis.phi(nb, np.array([-1.0]))[:, 0], rtol=1e-14, atol=1e-14)
    rng = np.random.default_rng(7)
    FA = rng.standard_normal(2 * QP + 8 * QPf)
    Fx = FA[:QP].reshape(npj, npj, npj)              # [pt, py, px]
    Fy = FA[QP:2 * QP].reshape(npj, npj, npj)
    own = [FA[2 * QP + f * QPf:2 * QP + (f + 1) * QPf].reshape(npj, npj) for f in range(4)]
    nbr = [FA[2 * QP + (4 + f) * QPf:2 * QP + (5 + f) * QPf].reshape(npj, npj) for f in range(4)]
    # the kernel's passes: Vx, Wy (x sums), H (face tangential sums), U (y sums and faces),
    # J (time sums); k = (a_k, y_k, x_k) with x fastest
    Vx = np.einsum("klp,typ->tykl", T1, Fx)
    Wy = np.einsum("klp,typ->tykl", T0, Fy)
    H = [np.einsum("klp,tp->tkl", T0, own[f]) for f in range(4)]
    U = (np.einsum("abp,tpkl->tabkl", T0, Vx) + np.einsum("abp,tpkl->tabkl", T1, Wy)
         + np.einsum("k,l,tab->tabkl", ep, ep, H[0]) + np.einsum("k,l,tab->tabkl", em, em, H[1])
         + np.einsum("a,b,tkl->tabkl", ep, ep, H[2]) + np.einsum("a,b,tkl->tabkl", em, em, H[3]))
    J = np.einsum("cdt,tabkl->cakdbl", T0, U).reshape(thT, thT)
    npair = thT * thT
    ref = np.zeros((npair, 2 * QP + 8 * QPf))
    for dd in range(2):
        ref[:, dd * QP:(dd + 1) * QP] = tb.beta[dd].reshape(npair, QP)
    for f in range(4):
        dd, side = f >> 1, (+1, -1)[f & 1]
        o = 2 * QP + f * QPf
        ref[:, o:o + QPf] = tb.gamma[dd][(side, side)].reshape(npair, QPf)
    scale = np.abs(ref).max() * np.abs(FA).max()
    np.testing.assert_allclose(J, (ref @ FA).reshape(thT, thT), rtol=0, atol=1e-12 * scale)
    # neighbour blocks: this cell's trace on its side of face f, the neighbour's on the other
    for f in range(4):
        dd, si = f >> 1, f & 1
        side = (+1, -1)[si]
        trk, trl = (em, ep) if si else (ep, em)
        K = np.einsum("cdt,tab->cdab", T0, np.einsum("abp,tp->tab", T0, nbr[f]))
        if dd == 0:   # normal x, tangential y
            N = np.einsum("k,l,cdab->cakdbl", trk, trl, K)
        else:         # normal y, tangential x
            N = np.einsum("a,b,cdkl->cakdbl", trk, trl, K)
        N = N.reshape(thT, thT)
        o = 2 * QP + (4 + f) * QPf
        G = tb.gamma[dd][(side, -side)].reshape(npair, QPf)
        np.testing.assert_allclose(N, (G @ FA[o:o + QPf]).reshape(thT, thT), rtol=0,
                                   atol=1e-12 * scale)


def test_elimination_plan_solves_region_system(exe):
    r = subprocess.run([exe, "plan"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "slots 43" in r.stdout        # 9 diagonal + 24 neighbour + 10 fill blocks
