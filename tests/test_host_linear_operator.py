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


def _operator(exe, d, M, nu, tmp_path):
    path = str(tmp_path / "P.txt")
    nu3 = list(nu) + [0.0] * (3 - len(nu))
    subprocess.run([exe, str(d), str(M)] + [repr(float(v)) for v in nu3] + [path], check=True,
                   capture_output=True)
    lines = open(path).read().split()
    lo, cnt = [int(v) for v in lines[0:3]], [int(v) for v in lines[3:6]]
    n, size = int(lines[6]), int(lines[7])
    P = np.array([float(v) for v in lines[8:8 + size]])
    return lo, cnt, n, P


CASES = [
    (1, 3, (0.9,)), (1, 6, (-0.45,)), (1, 2, (0.0,)),
    (2, 1, (0.35, 0.175)), (2, 3, (0.35, 0.175)), (2, 2, (-0.3, 0.2)), (2, 3, (0.3, -0.7)),
    (2, 2, (0.0, -0.4)), (3, 1, (0.3, 0.21, 0.09)), (3, 2, (0.3, -0.21, 0.0)),
    (3, 1, (-0.6, -0.6, 0.6)),
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
