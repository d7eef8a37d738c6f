"""ridg_l2_error_noalloc: the L2-error diagnostic for callers that cannot allocate device
memory (it uses a fixed scratch array inside the library instead of cudaMalloc).  It must
agree with the ordinary entry point, call after call, since every call reuses that array.
This file is collected last so that a failure here cannot hide any other test."""
import numpy as np
import pytest

from paper_2101_01231_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2101_01231_gb300 import ridg as R

    w = I.workload("adv2d_n256_q3", n=(48, 40))
    s = R.Solver(2, w["n"], w["M"], vel=w["vel"], cfl=w["cfl"], lo=w["lo"], hi=w["hi"])
    s.set_state(I.initial_state(w))
    s.set_final_time(0.25)
    Xd = torch.from_numpy(I.exact_coefficients(w, 0.25)).cuda()
    qd = torch.empty(s.cells, s.theta_s, dtype=torch.float64, device="cuda")
    return torch, R, w, s, Xd, qd


def test_noalloc_l2_error_matches_handle_entry_point():
    torch, R, w, s, Xd, qd = _setup()
    for call in range(2):
        # a different state for each call: the shared scratch must not carry anything over
        s.step(3)
        s.sync()
        s.get_state(qd)
        torch.cuda.synchronize()
        ref = s.l2_error(Xd)
        got = R.ridg_l2_error_noalloc(qd, Xd, s.cells, 1, 2, w["M"])
        assert abs(got - ref) <= 1e-12 * ref, (call, got, ref)
    # on a stream of the caller's: same value, and no device memory taken by the call
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    free0 = torch.cuda.mem_get_info()[0]
    got = R.ridg_l2_error_noalloc(qd, Xd, s.cells, 1, 2, w["M"], stream=st)
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(got - ref) <= 1e-12 * ref, (got, ref)
    assert free1 == free0, (free0, free1)
    # a size beyond the fixed scratch is refused before any work is done (the arrays are
    # sized to match, so only the limit can refuse it)
    big = 65536 * 256 + 1
    qb = torch.zeros(big, 1, dtype=torch.float64, device="cuda")
    xb = torch.zeros(big, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RidgError) as e:
        R.ridg_l2_error_noalloc(qb, xb, big, 1, 2, 0)
    assert e.value.status == R.RIDG_ETOOBIG
    # arrays that do not match the sizes never reach the library
    with pytest.raises(ValueError):
        R.ridg_l2_error_noalloc(qd, Xd, s.cells + 1, 1, 2, w["M"])
    s.close()


def test_noalloc_refuses_a_capturing_stream():
    torch, R, w, s, Xd, qd = _setup()
    s.get_state(qd)
    torch.cuda.synchronize()
    ref = R.ridg_l2_error_noalloc(qd, Xd, s.cells, 1, 2, w["M"])  # device set-up done
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        g.capture_begin()
        try:
            with pytest.raises(R.RidgError) as e:
                R.ridg_l2_error_noalloc(qd, Xd, s.cells, 1, 2, w["M"], stream=st)
            qd.mul_(1.0)  # some captured work, so that the graph is not empty
        finally:
            g.capture_end()  # the refusal left the caller's capture intact
    assert e.value.status == R.RIDG_ESTATE
    g.replay()
    torch.cuda.synchronize()
    got = R.ridg_l2_error_noalloc(qd, Xd, s.cells, 1, 2, w["M"])
    assert abs(got - ref) <= 1e-12 * ref, (got, ref)
    s.close()
