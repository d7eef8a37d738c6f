"""ridg_l2_error_noalloc: the L2-error diagnostic for callers that cannot allocate device
memory (it uses a fixed scratch array inside the library instead of cudaMalloc).  It must
agree with the ordinary entry point, call after call, since every call reuses that array.
This file is collected last so that a failure here cannot hide any other test."""
import numpy as np
import pytest

from paper_2101_01231_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_l2_error_matches_handle_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2101_01231_gb300 import ridg as R

    w = I.workload("adv2d_n256_q3", n=(48, 40))
    s = R.Solver(2, w["n"], w["M"], vel=w["vel"], cfl=w["cfl"], lo=w["lo"], hi=w["hi"])
    q0 = I.initial_state(w)
    X = I.exact_coefficients(w, 0.25)
    Xd = torch.from_numpy(X).cuda()
    qd = torch.empty(s.cells, s.theta_s, dtype=torch.float64, device="cuda")
    s.set_state(q0)
    s.set_final_time(0.25)
    for call in range(2):
        # a different state for each call: the shared scratch must not carry anything over
        s.step(3)
        s.sync()
        s.get_state(qd)
        torch.cuda.synchronize()
        ref = s.l2_error(Xd)
        got = R.ridg_l2_error_noalloc(qd, Xd, s.cells, 1, 2, w["M"])
        assert abs(got - ref) <= 1e-12 * ref, (call, got, ref)
    # a size beyond the fixed scratch is refused before any work is done
    with pytest.raises(R.RidgError) as e:
        R.ridg_l2_error_noalloc(qd, Xd, 65536 * 256 + 1, 1, 2, w["M"])
    assert e.value.status == R.RIDG_ETOOBIG
    s.close()
