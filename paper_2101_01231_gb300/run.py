"""Run a named workload through the C ABI and report device times.

    python -m paper_2101_01231_gb300.run --workload euler2d_n512_q2 --mesh 64 64 \\
        --precision mixed_fp32 --steps 2

Sets the seeded synthetic initial state of the workload (optionally on another mesh or
degree), takes --warmup untimed steps and --steps steps with per-kernel CUDA-event timing
(ridg_profile_step), and prints one JSON line with the times and the Newton statistics.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import inputs as I
from . import ridg as R

PRECISIONS = {"fp64": R.RIDG_PREC_FP64, "mixed_bf16": R.RIDG_PREC_MIXED_BF16,
              "mixed_fp16": R.RIDG_PREC_MIXED_FP16,
              "mixed_fp32": R.RIDG_PREC_MIXED_FP32, "mixed_tf32": R.RIDG_PREC_MIXED_TF32}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--workload", required=True, choices=sorted(I.WORKLOADS))
    p.add_argument("--mesh", type=int, nargs="+", help="cells per dimension (override)")
    p.add_argument("--order", type=int, help="polynomial degree M (override)")
    p.add_argument("--precision", default="fp64", choices=sorted(PRECISIONS))
    p.add_argument("--slices", type=int, default=0, help="digit slices of the mixed BF16 path")
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=0)
    p.add_argument("--autotune", action="store_true",
                   help="run the library's autotuner on the state before the steps")
    a = p.parse_args(argv)
    over = {}
    if a.mesh:
        over["n"] = tuple(a.mesh)
    if a.order is not None:
        over["M"] = a.order
    w = I.workload(a.workload, **over)
    s = R.Solver(w["dim"], w["n"], w["M"], flux=w["flux"], vel=w.get("vel", (0.0, 0.0, 0.0)),
                 cfl=w["cfl"], lo=w["lo"], hi=w["hi"], gamma=w.get("gamma", 1.4),
                 precision=PRECISIONS[a.precision], slices=a.slices)
    s.set_state(I.initial_state(w))
    if a.autotune:
        s.autotune()
    if a.warmup:
        s.profile_step(a.warmup)
    prof = s.profile_step(a.steps)
    info = s.info()
    tuning = s.tuning()
    s.close()
    cells = int(np.prod(w["n"]))
    print(json.dumps({"workload": a.workload, "mesh": list(w["n"]), "order": w["M"],
                      "precision": a.precision, "steps": a.steps, **prof,
                      "dof_per_s": cells * info["m"] * info["theta_s"] / (prof["step_ms"] * 1e-3),
                      "newton_iters_total": info["newton_iters_total"],
                      "newton_iters_max": info["newton_iters_max"],
                      "newton_unconverged": info["newton_unconverged"], "tuning": tuning}))


if __name__ == "__main__":
    main()
