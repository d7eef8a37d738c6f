"""A mesh sharded into slabs along its slowest axis (ridg_shard_*, the domain decomposition of
Sec. 5 with one two-layer halo exchange per step) against the unsharded step: the FP64 path
bit for bit (every owned cell reads the same operands in the same order), the mixed path
to its tolerance (each slab takes its own digit exponent)."""
import numpy as np
import pytest

from paper_2101_01231_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2101_01231_gb300 import ridg
    return ridg


CASES = [
    # dim, mesh, degree, velocity, slabs
    (3, (8, 6, 9), 2, (1.0, 0.7, 0.3), 3),
    (3, (7, 5, 10), 1, (0.4, -0.9, -0.6), 4),
    (3, (6, 6, 8), 2, (0.5, 0.8, 0.0), 2),        # no flux along the slab axis: no halo
    (2, (13, 11), 3, (1.0, 0.5), 2),
    (2, (9, 12), 2, (-0.7, -1.0), 5),
    (1, (20,), 3, (1.0,), 3),
    (3, (6, 5, 7), 1, (1.0, 0.5, 0.25), 1),       # one slab: its own periodic halo
]


@pytest.mark.parametrize("dim,n,M,vel,count", CASES)
def test_sharded_fp64_step_is_bit_identical(R, dim, n, M, vel, count):
    rng = np.random.default_rng(sum(n) + count)
    q = rng.standard_normal((int(np.prod(n)), (M + 1) ** dim))
    s = R.Solver(dim, n, M, vel=vel, cfl=0.3)
    s.set_state(q)
    s.step(4)
    s.sync()
    ref = s.get_state()
    s.close()
    sh = R.Shard(dim, n, M, vel, 0.3, count)
    sh.set_state(q)
    sh.step(3)
    sh.step(1)
    sh.sync()
    out = np.empty_like(q)
    sh.get_state(out)
    sh.close()
    assert np.array_equal(out, ref)


def test_sharded_mixed_step(R):
    w = I.workload("adv3d_n96_q2", n=(16, 16, 12))
    q = I.initial_state(w)
    s = R.Solver(3, w["n"], w["M"], vel=w["vel"], cfl=w["cfl"])
    s.set_state(q)
    s.step(5)
    s.sync()
    ref = s.get_state()
    s.close()
    sh = R.Shard(3, w["n"], w["M"], w["vel"], w["cfl"], 3, precision=R.RIDG_PREC_MIXED_BF16,
                 slices=6)
    sh.set_state(q)
    sh.step(5)
    sh.sync()
    out = np.empty_like(q)
    sh.get_state(out)
    sh.close()
    assert float(np.abs(out - ref).max() / np.abs(ref).max()) < 5e-12


def test_shard_rejects_thin_slabs_and_nonlinear(R):
    with pytest.raises(R.RidgError):
        R.Shard(3, (6, 6, 5), 1, (1.0, 1.0, 1.0), 0.3, 3)     # a slab of one layer
