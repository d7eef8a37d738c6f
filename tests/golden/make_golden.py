"""Write the oracle's final-time accuracy figures used as the equal-accuracy reference.

Runs only the oracle (oracle/) on the seeded inputs (paper_2101_01231_gb300/inputs.py) and
stores, per workload, the number of steps, dt and the relative L2 error of eq. l2relerror
against the exact solution at the final time.  For the noisy 3D data (whose exact solution
is the noisy piecewise polynomial carried by a t) the error is integrated exactly on the
sub-box overlaps (inputs.shifted_polynomial_error), and the final coefficients of a seeded
sample of cells are stored beside it (<key>_cells.npz) for element-wise parity.  Usage:

    python tests/golden/make_golden.py [name ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import error as oerr  # noqa: E402
from oracle import linear as OL  # noqa: E402
from paper_2101_01231_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_accuracy.json")

RUNS = {
    # name: (workload, overrides, final time)
    "adv1d_n64_q3": ("adv1d_n64_q3", {}, 1.0),
    "adv2d_n256_q3": ("adv2d_n256_q3", {}, 1.0),
    # noise-free variant of the 3D workload on a 24^3 mesh (same degree, velocity, CFL)
    "adv3d_n24_q2_sin": ("adv3d_n96_q2", {"n": (24, 24, 24), "ic": "sin"}, 1.0),
    # the stated 3D data (product of sines + seeded 1e-3 noise) on a 24^3 mesh
    "adv3d_n24_q2_noise": ("adv3d_n96_q2", {"n": (24, 24, 24)}, 1.0),
}
SAMPLE_CELLS = 256
# nonlinear flux (the pooled oracle, tests/oracle_pool.py): the Euler vortex at the config's
# degree on a 32^2 mesh to t = 1, and the Burgers ensemble capped at 16^2 cells per instance,
# each instance to half its shock time in a common number of steps
NL_RUNS = ("euler2d_n32_q2", "burgers_ens16")


def run(key):
    name, over, T = RUNS[key]
    w = I.workload(name, **over)
    dt, nt = OL.advection_time_step(w, T=T)
    q = I.initial_state(w)
    t0 = time.time()
    q0 = q
    q = OL.run(q, w, dt, nt)
    extra = {}
    if w.get("ic") == "sin+noise":
        err = I.shifted_polynomial_error(w, q0, q, T)
        extra["cells_file"] = _sample(q, key)
    else:
        err = oerr.l2_relative_error(q, I.exact_coefficients(w, T), w["M"], w["dim"])
    return dict(workload=name, overrides={k: list(v) if isinstance(v, tuple) else v
                                          for k, v in over.items()},
                T=T, steps=nt, dt=dt, l2_error=err, oracle_seconds=round(time.time() - t0, 1),
                **extra)


def _sample(q, key):
    cells = np.sort(np.random.default_rng(0).choice(q.shape[0], min(SAMPLE_CELLS, q.shape[0]),
                                                    replace=False))
    np.savez_compressed(os.path.join(os.path.dirname(OUT), f"{key}_cells.npz"), cells=cells,
                        q=q[cells])
    return f"{key}_cells.npz"


def burgers_ensemble_setup(cap=16):
    """The 64 ensemble instances capped at cap^2 cells, T_i = t_shock_i / 2, and the common
    step count N (each instance's dt_i = T_i / N, within its CFL step)."""
    from oracle import linear as OL
    from oracle import nonlinear as ONL
    ens = [dict(w, n=(min(w["n"][0], cap), min(w["n"][1], cap))) for w in I.burgers_ensemble()]
    Ts = [0.5 * I.burgers_shock_time(w) for w in ens]
    N = 0
    for w, T in zip(ens, Ts):
        dt_cfl, _ = OL.time_step(w, ONL.max_speed(I.initial_state(w), w))
        N = max(N, int(np.ceil(T / dt_cfl - 1e-9)))
    return ens, Ts, N


def run_nl(key):
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import linear as OL
    from oracle import nonlinear as ONL
    from oracle_pool import Pool
    t0 = time.time()
    with Pool() as pool:
        if key == "euler2d_n32_q2":
            w = I.workload("euler2d_n512_q2", n=(32, 32))
            q0 = I.initial_state(w)
            dt, nt = OL.time_step(w, ONL.max_speed(q0, w), 1.0)
            q, unconv = pool.run(q0, w, dt, nt)
            err = oerr.l2_relative_error(q, I.exact_coefficients(w, 1.0), w["M"], 2, m=4)
            return dict(workload="euler2d_n512_q2", overrides={"n": [32, 32]}, T=1.0, steps=nt,
                        dt=dt, l2_error=err, unconverged_region_steps=unconv,
                        cells_file=_sample(q, key), oracle_seconds=round(time.time() - t0, 1))
        ens, Ts, N = burgers_ensemble_setup()
        # the oracle's reference: the first four instances of each degree (16 of 64; the
        # Q3 / Q4 Newton solves of numpy make all 64 a matter of hours)
        pick = [i for m in (1, 2, 3, 4) for i in [j for j, w in enumerate(ens) if w["M"] == m][:4]]
        errs, unc = [], 0
        for i in pick:
            w, T = ens[i], Ts[i]
            q, u = pool.run(I.initial_state(w), w, T / N, N)
            unc += u
            errs.append(oerr.l2_relative_error(q, I.exact_coefficients(w, T), w["M"], 2))
            print(f"  instance {i}: M={w['M']} err={errs[-1]:.4e}", flush=True)
        return dict(workload="burgers_ensemble capped at 16^2", steps=N, T=Ts, instances=pick,
                    l2_error=errs, unconverged_region_steps=unc,
                    oracle_seconds=round(time.time() - t0, 1))


def main(keys):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for k in keys:
        data[k] = run_nl(k) if k in NL_RUNS else run(k)
        print(k, data[k], flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(RUNS) + list(NL_RUNS))
