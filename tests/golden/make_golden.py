"""Write the oracle's final-time accuracy figures used as the equal-accuracy reference.

Runs only the oracle (oracle/) on the seeded inputs (paper_2101_01231_gb300/inputs.py) and
stores, per workload, the number of steps, dt and the relative L2 error of eq. l2relerror
against the exact solution at the final time.  Usage:

    python tests/golden/make_golden.py [name ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

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
}


def run(key):
    name, over, T = RUNS[key]
    w = I.workload(name, **over)
    dt, nt = OL.advection_time_step(w, T=T)
    q = I.initial_state(w)
    t0 = time.time()
    q = OL.run(q, w, dt, nt)
    err = oerr.l2_relative_error(q, I.exact_coefficients(w, T), w["M"], w["dim"])
    return dict(workload=name, overrides={k: list(v) if isinstance(v, tuple) else v
                                          for k, v in over.items()},
                T=T, steps=nt, dt=dt, l2_error=err, oracle_seconds=round(time.time() - t0, 1))


def main(keys):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for k in keys:
        data[k] = run(k)
        print(k, data[k], flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(RUNS))
