"""The autotuner (ridg_autotune): it times the launch choices on the handle's own state,
keeps the fastest, puts the state back, and later handles of the same configuration read
the choice from the cache (also written to a file)."""
import numpy as np
import pytest

from oracle import linear as OL
from paper_2101_01231_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2101_01231_gb300 import ridg
    return ridg


def test_autotune_3d_mixed(R, tmp_path):
    w = I.workload("adv3d_n96_q2", n=(32, 32, 24))
    mk = lambda: R.Solver(3, w["n"], w["M"], vel=w["vel"], cfl=w["cfl"],
                          precision=R.RIDG_PREC_MIXED_BF16, slices=4)
    s = mk()
    q0 = I.initial_state(w)
    s.set_state(q0)
    path = str(tmp_path / "tune.txt")
    s.autotune(path)
    t = s.tuning()
    assert t["gemm3_slots"] in (3, 4, 5, 6, 8) and t["corr3_block"] in (64, 128, 256)
    assert np.array_equal(s.get_state(), q0) and s.info()["steps"] == 0   # state put back
    # the tuned handle still steps correctly
    dt = s.info()["dt"]
    s.step(2)
    s.sync()
    ref = OL.run(q0, w, dt, 2)
    # four slices: up to 2^-32 x 64 of the state's scale per step (the bound the other 3D
    # tests use at S = 4)
    assert float(np.abs(s.get_state() - ref).max() / np.abs(ref).max()) < 2 * 2.0 ** -32 * 64
    s.close()
    # a new handle of the same configuration reads the choice; the file holds it
    s2 = mk()
    assert s2.tuning() == t
    s2.close()
    assert f"corr3.block nb3 S4 {t['corr3_block']}" in open(path).read()


def test_autotune_newton_grid(R):
    w = dict(I.burgers_ensemble(1)[0], n=(24, 20), M=2)
    s = R.Solver(2, w["n"], w["M"], flux="burgers", cfl=w["cfl"],
                 precision=R.RIDG_PREC_MIXED_TF32)
    q0 = I.initial_state(w)
    s.set_state(q0)
    g0 = s.tuning()["newton_grid"]
    s.autotune()
    g = s.tuning()["newton_grid"]
    assert 1 <= g <= g0
    assert np.array_equal(s.get_state(), q0)
    s.step(1)
    assert s.sync() == R.RIDG_OK
    s.close()
    s2 = R.Solver(2, w["n"], w["M"], flux="burgers", cfl=w["cfl"],
                  precision=R.RIDG_PREC_MIXED_TF32)
    assert s2.tuning()["newton_grid"] == g
    s2.close()
