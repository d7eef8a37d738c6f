#!/usr/bin/env python
"""RIDG step throughput on one GB300 (element-DOF updates/s).

Headline workload: 3D linear advection with velocity (1, 0.7, 0.3) on the periodic unit
cube, 96^3 cells, tensor Q2 (27 spatial / 81 space-time coefficients), 3 x 3 x 3 regions,
u0 = product of sines plus seeded U(-1e-3, 1e-3) noise on every coefficient, CFL 0.30,
final time 1 (320 steps).  A step is one prediction + correction over the whole mesh.
Inputs are seeded synthetic data resident in HBM; the 191 MB state is larger than the
129 MB L2, and a 256 MB buffer is rewritten before every timed step as well.

The timed arm reports the mixed BF16 tensor-core path at the fewest digit slices whose L2
error against the exact solution at t = 1 (the noisy piecewise polynomial carried by a t,
integrated exactly on the sub-box overlaps) is within 1.05x of the FP64 path's, with the
FP64 path beside it, the 2D 256^2 Q3 workload as an extra object, and the oracle on the
host cores.  --impl reference times the oracle alone.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "adv3d_n96_q2"
WORKLOAD_2D = "adv2d_n256_q3"
T_FINAL = 1.0


def upwind_cells(w):
    """Region cells a linear prediction reads: {-1, 0} or {0, +1} along each dimension with a
    nonzero velocity component (upstream of the centre), {0} along the others."""
    return 2 ** sum(1 for v in list(w["vel"])[: w["dim"]] if v != 0)


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="auto", choices=["auto", "fp64", "mixed"])
    p.add_argument("--slices", type=int, default=0)
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--newton-steps", type=int, default=1,
                   help="timed steps of the Newton path (0: skip it)")
    p.add_argument("--paper1d", type=int, default=1,
                   help="the paper's 1D table (degrees 3-11) on the GPU (0: skip)")
    p.add_argument("--paper2d", type=int, default=1,
                   help="run the paper's 2D study (60^2 bump, degrees 3 and 5; 0 skips it)")
    p.add_argument("--paper3d", type=int, default=1,
                   help="run the paper's 3D study (48^3 bump, degrees 3 and 5; 0 skips it)")
    p.add_argument("--adv1d-reps", type=int, default=20,
                   help="whole 1D runs to T = 1 timed (0: skip the 1D section)")
    p.add_argument("--ensemble-steps", type=int, default=1,
                   help="full-size Burgers-ensemble steps timed (0: skip; ~45 s per step)")
    p.add_argument("--autotune", type=int, default=1,
                   help="run the library's autotuner (ridg_autotune) before timing (0: defaults)")
    p.add_argument("--adv2d-steps", type=int, default=200,
                   help="timed steps of the 2D 256^2 Q3 workload beside the headline (0: skip)")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device="cpu"):
    """The largest of every rank's x (ws > 1: an all-reduce MAX over the process group)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(items, rank, ws):
    """One rank's round-robin share of independent units (the ensemble's instances)."""
    return list(items)[rank::ws]


def _golden():
    p = os.path.join(ROOT, "tests", "golden", "oracle_accuracy.json")
    return json.load(open(p)) if os.path.exists(p) else {}


# ---------------------------------------------------------------------------------------
# the oracle on the host (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------------------
def cpu_oracle(w, seconds, steps=None):
    """Time oracle steps of the full workload until `seconds` of CPU work (or `steps`)."""
    from oracle import linear as OL
    from paper_2101_01231_gb300 import inputs as I
    q = I.initial_state(w)
    dt, _ = OL.advection_time_step(w, T=T_FINAL)
    n = 0
    t0 = time.perf_counter()
    while True:
        q = OL.step(q, w, dt)
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (steps is None and el >= seconds):
            break
    cells = int(np.prod(w["n"]))
    dof = cells * (w["M"] + 1) ** w["dim"]
    return dict(value=dof * n / el, unit="element-DOF updates/s", cores=os.cpu_count(),
                kind="oracle", steps=n, seconds=round(el, 3),
                sample=f"{n} full oracle steps of {w['name']} ({cells} cells, region LU solves, "
                       f"numpy/scipy on all host cores)")


def cpu_oracle_sampled(w, q, nsample=4096, seed=0):
    """One oracle step of w as it stands, estimated from timed parts: the region system's
    factorisation (once per step), the region solves of a seeded sample of cells scaled to
    all cells, and the correction of Sec. 2.3 timed on the whole mesh."""
    from oracle import linear as OL
    cells = int(np.prod(w["n"]))
    thS = (w["M"] + 1) ** w["dim"]
    dt, _ = OL.advection_time_step(w, T=T_FINAL)
    sample = np.sort(np.random.default_rng(seed).choice(cells, size=min(nsample, cells),
                                                        replace=False))
    t0 = time.perf_counter()
    OL.region_solver(w["dim"], w["M"], OL.nu_of(w, dt))
    t_factor = time.perf_counter() - t0
    t0 = time.perf_counter()
    W = OL.predict_cells(q, w, dt, sample)     # its own factorisation + the sample's solves
    t_pred = time.perf_counter() - t0
    Wbar = np.zeros((cells, thS))
    Wbar[sample] = W[:, :thS]
    t0 = time.perf_counter()
    OL.correct(q, Wbar, w, dt)
    t_corr = time.perf_counter() - t0
    per_step = t_factor + max(t_pred - t_factor, 0.0) / len(sample) * cells + t_corr
    dof = cells * thS
    return dict(value=dof / per_step, unit="element-DOF updates/s", cores=os.cpu_count(),
                kind="oracle", seconds=round(t_factor + t_pred + t_corr, 3),
                extrapolated_step_s=per_step,
                sample=f"one oracle step of {w['name']} ({cells} cells): the factorisation, "
                       f"the region solves of {len(sample)} seeded cells scaled to all cells, "
                       f"and the correction on the whole mesh (numpy/scipy, all host cores)")


def run_reference(args):
    """The oracle on the host cores for the headline workload: each step a full oracle step
    (2D) or, in 3D where a full oracle step takes minutes, one oracle step estimated from a
    seeded sample of 1024 region solves scaled to the mesh plus the correction of the whole
    mesh (cpu_oracle_sampled); at most about two minutes of host time in all."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2101_01231_gb300 import inputs as I
    w = I.workload(args.workload)
    cells = int(np.prod(w["n"]))
    dof = cells * (w["M"] + 1) ** w["dim"]
    sampled = w["dim"] == 3
    q = I.initial_state(w)

    def one(seed):
        if sampled:
            r = cpu_oracle_sampled(w, q, nsample=1024, seed=seed)
            return r["extrapolated_step_s"], r["seconds"]
        r = cpu_oracle(w, 0, steps=1)
        return r["seconds"], r["seconds"]

    for i in range(max(1, min(args.warmup, 3))):
        one(1000 + i)  # warm-up (tables, BLAS threads)
    t_step, t_wall, n_all = 0.0, 0.0, 0
    for i in range(args.steps):
        ts, tw = one(i)
        t_step += ts
        t_wall += tw
        n_all += 1
        if t_wall > 120:
            break
    value = dof * n_all / t_step
    sample = (f"{n_all} oracle steps, each estimated from 1024 seeded region solves scaled to "
              f"{cells} cells plus the correction of the whole mesh" if sampled
              else f"{n_all} full oracle steps")
    line = {
        "impl": "reference", "metric": "element-DOF updates/s per RIDG step",
        "value": value, "unit": "element-DOF updates/s", "n_gpus": ws, "steps": n_all,
        "warmup": 1, "ms_per_step": 1e3 * t_step / n_all, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "cells": cells, "order": w["M"], "steps_to_T": None},
        "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": value,
                         "unit": "element-DOF updates/s", "sample": sample + " (host cores)"},
        "e2e": {"value": value, "unit": "element-DOF updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def adv1d_section(R, I, reps):
    """1D advection, 64 cells, Q3, FP64, to t = 1: the whole run (one captured graph of all
    its steps) timed with CUDA events, per step in ns; its L2 error against the exact
    solution and the oracle's, and the oracle's own run on the host."""
    import torch
    from oracle import error as OE
    from oracle import linear as OL
    w = I.workload("adv1d_n64_q3")
    q0 = I.initial_state(w)
    s = R.Solver(1, w["n"], w["M"], vel=w["vel"], cfl=w["cfl"], lo=w["lo"], hi=w["hi"])
    s.set_state(q0)
    nt = s.set_final_time(T_FINAL)
    s.step(nt)                                  # warm-up (captures the nt-step graph)
    s.sync()
    exact = I.exact_coefficients(w, T_FINAL)
    err = s.l2_error(exact)
    dt = s.info()["dt"]
    times = []
    for _ in range(reps):
        s.set_state(q0)
        s.set_final_time(T_FINAL)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        s.step(nt)
        b.record(s.stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    s.close()
    ms = float(np.median(times))
    t0 = time.perf_counter()
    qo = OL.run(q0, w, dt, nt)
    t_or = time.perf_counter() - t0
    err_or = OE.l2_relative_error(qo, exact, w["M"], 1)
    cells, thS = int(np.prod(w["n"])), w["M"] + 1
    return {"workload": w["name"], "steps_to_T": nt, "run_ms": ms, "ns_per_step": ms / nt * 1e6,
            "value": cells * thS * nt / (ms * 1e-3), "unit": "element-DOF updates/s",
            "roofline": None, "bound": "launch / latency (2 KB of state)",
            "l2_error": err, "l2_error_oracle": err_or,
            "cpu_oracle": {"kind": "oracle", "cores": 1, "seconds_per_run": t_or,
                           "value": cells * thS * nt / t_or, "unit": "element-DOF updates/s",
                           "sample": f"the whole run ({nt} steps)"}}


def ensemble_section(R, I, steps, cpu_cells, rank=0, ws=1):
    """The batched Burgers ensemble (64 instances, N ~ U{64..512}, Q1-Q4, seeded Fourier data)
    advanced by ridg_batch_step: one captured graph per step holding one persistent Newton
    launch per degree over all the instances of that degree, then the corrections; TF32
    block updates with the FP64 residual.  Warm-up on the same ensemble capped at 64 x 64
    (the same kernels), then `steps` full-size steps timed with CUDA events on the batch's
    stream; the oracle's Newton prediction on a sample of cells per degree, extrapolated."""
    import torch
    from oracle import linear as OL
    from oracle import nonlinear as ONL
    ens_all = I.burgers_ensemble()
    ens = shard(ens_all, rank, ws)  # N GPUs: the instances round-robin over the ranks
    stream = torch.cuda.Stream()
    opt = R.make_options(precision=R.RIDG_PREC_MIXED_TF32, stream=stream.cuda_stream)

    def batch(ws):
        b = R.ridg_batch_create([R.make_mesh(2, w["n"]) for w in ws], [w["M"] for w in ws],
                                R.make_flux("burgers"), ws[0]["cfl"], opt)
        for i, w in enumerate(ws):
            R.ridg_set_state(R.ridg_batch_instance(b, i), I.initial_state(w))
        return b

    if AUTOTUNE[0]:
        # the Newton grid per degree, timed on a 128^2 copy of the first instance of each
        # degree; the batch's instances read the choices at ridg_batch_create
        for m in sorted({w["M"] for w in ens}):
            wt = dict(next(x for x in ens if x["M"] == m), n=(128, 128))
            st = R.Solver(2, wt["n"], m, flux="burgers", cfl=wt["cfl"],
                          precision=R.RIDG_PREC_MIXED_TF32)
            st.set_state(I.initial_state(wt))
            st.autotune()
            st.close()
    small = [dict(w, n=(min(w["n"][0], 64), min(w["n"][1], 64))) for w in ens]
    b = batch(small)
    R.ridg_batch_step(b, 1)
    R.ridg_batch_sync(b)
    if AUTOTUNE[0]:
        # the schedule (the whole ensemble in two launches, or a launch per degree and per
        # instance), timed on the capped ensemble; the full batch reads the choice
        R.ridg_batch_autotune(b)
    R.ridg_batch_destroy(b)
    b = batch(ens)
    sched = R.ridg_batch_schedule(b)
    times, status = [], []
    for _ in range(steps):
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        R.ridg_batch_step(b, 1)
        a1.record(stream)
        status.append(R.ridg_batch_sync(b))
        times.append(a0.elapsed_time(a1))
    infos = [R.ridg_info(R.ridg_batch_instance(b, i)) for i in range(len(ens))]
    R.ridg_batch_destroy(b)
    ms = max_over_ranks(float(np.mean(times)), ws, "cuda")
    dof = sum(int(np.prod(w["n"])) * (w["M"] + 1) ** 2 for w in ens_all)
    # algorithmic work of the block eliminations: 118 b^3 flop per factorisation, b = theta_T
    flops = sum(118.0 * (w["M"] + 1) ** 9 * inf["newton_iters_total"] for w, inf in zip(ens, infos))
    ach = flops / (ms * 1e-3) / 1e12  # per GPU: this rank's instances over the step time
    out = {"workload": "burgers_ensemble_64", "instances": len(ens_all),
           "scaling": "strong: the 64 instances round-robin over the ranks",
           "cells": sum(int(np.prod(w["n"])) for w in ens_all),
           "cells_per_degree": {str(m): sum(int(np.prod(w["n"])) for w in ens_all if w["M"] == m)
                                for m in (1, 2, 3, 4)},
           "precision": "mixed_tf32", "steps": steps, "ms_per_step": ms,
           "value": dof / (ms * 1e-3), "unit": "element-DOF updates/s",
           "schedule": ("the whole ensemble's Newton prediction in one launch (every degree's "
                        "regions, highest degree first) + every instance's correction in one"
                        if sched["schedule"] == 1 else
                        "one Newton launch per degree + one correction per instance"),
           "launches_per_step": sched["launches_per_step"],
           "newton_unconverged": sum(inf["newton_unconverged"] for inf in infos),
           "status": [int(x) for x in status],
           "roofline": {"bound": "alu", "kernel": "newton_kernel (all degrees)",
                        "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": ach / FP32_PEAK_TFLOPS, "traffic": None,
                        "peak_source": "nominal: FMA pipes x 2 flop x 2.07 GHz"}}
    out["accuracy"] = ensemble_accuracy(R, I, R.RIDG_PREC_MIXED_TF32)
    # the oracle: per-cell Newton prediction time per degree (a 32 x 32 copy of the first
    # instance of each degree), extrapolated to the ensemble's cells
    if rank != 0:
        return out
    per = {}
    for m in (1, 2, 3, 4):
        w = dict(next(x for x in ens_all if x["M"] == m), n=(32, 32))
        q = I.initial_state(w)
        dt, _ = OL.time_step(w, ONL.max_speed(q, w))
        k = cpu_cells if m < 3 else 2
        t0 = time.perf_counter()
        ONL.newton_predict(q, w, dt, cells=np.arange(k))
        per[m] = (time.perf_counter() - t0) / k
    t_or = sum(int(np.prod(w["n"])) * per[w["M"]] for w in ens_all)
    out["cpu_oracle"] = {"kind": "oracle", "cores": os.cpu_count(),
                         "seconds_per_cell": {str(m): v for m, v in per.items()},
                         "value": dof / t_or, "unit": "element-DOF updates/s",
                         "sample": f"Newton predictions of {cpu_cells} cells (Q1, Q2) / 2 cells "
                                   "(Q3, Q4) per degree, extrapolated to the ensemble (numpy)"}
    return out


def paper1d_section(R, I):
    """The paper's own 1D study (table table:1D): RIDG at nu = 0.9 on the C-infinity bump of
    eq. adv1d, degrees 3 to 11 on the table's meshes, run to t = 1 (the paper states no final
    time) on the GPU -- each run one single-CTA launch -- with its L2 error, observed order
    (eq. Mratio), run time and quality = -log10(error x runtime) (eq. Quality); beside it the
    oracle's error and host run time, and the paper's printed CPU figures."""
    import torch
    from oracle import error as OE
    from oracle import linear as OL
    ref = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_1d_table.json")))

    def bump(x):
        r2 = (x - 0.5) ** 2
        out = np.zeros_like(x)
        m = r2 < 1.0 / 9.0
        out[m] = np.exp(1.0 / (r2[m] - 1.0 / 9.0))
        return out

    rows = {}
    for M in (3, 5, 7, 9, 11):
        meshes = ref["rows"][str(M)]["mesh"]
        r = {"mesh": meshes, "l2_error": [], "order": [None], "gpu_run_s": [], "quality": [],
             "l2_error_oracle": [], "oracle_run_s": [],
             "paper_l2_error": ref["rows"][str(M)]["error"],
             "paper_runtime_s": ref["runtime_s"][str(M)], "paper_quality": ref["quality"][str(M)]}
        for N in meshes:
            w = dict(flux="advection", dim=1, n=(N,), M=M, vel=(1.0,), lo=(0.0,), hi=(1.0,),
                     cfl=0.9)
            q0 = I.project_1d(bump, N, 0.0, 1.0, M + 1, nq=40)
            X = I.project_1d(bump, N, 0.0, 1.0, M + 2, nq=40)
            s = R.Solver(1, (N,), M, vel=(1.0,), cfl=0.9)
            s.set_state(q0)
            nt = s.set_final_time(T_FINAL)
            s.step(nt)                       # warm-up (captures the run's graph)
            s.sync()
            times = []
            for _ in range(5):
                s.set_state(q0)
                s.set_final_time(T_FINAL)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(s.stream)
                s.step(nt)
                b.record(s.stream)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b) * 1e-3)
            e = s.l2_error(X)
            dt = s.info()["dt"]
            s.close()
            t_gpu = float(np.median(times))
            t0 = time.perf_counter()
            qo = OL.run(q0, w, dt, nt)
            t_or = time.perf_counter() - t0
            r["l2_error"].append(e)
            r["gpu_run_s"].append(t_gpu)
            r["quality"].append(-np.log10(e * t_gpu))
            r["l2_error_oracle"].append(OE.l2_relative_error(qo, X, M, 1))
            r["oracle_run_s"].append(t_or)
        for k in range(1, len(meshes)):
            r["order"].append(OE.observed_order(r["l2_error"][k - 1], r["l2_error"][k],
                                                1 / meshes[k - 1], 1 / meshes[k]))
        rows[str(M)] = r
    return {"workload": "adv1d bump (eq. adv1d), nu = 0.9, t = 1", "precision": "fp64",
            "rows": rows}


def paper_bump_section(R, I, dim):
    """The paper's multi-dimensional advection studies on the GPU: RIDG on the C-infinity bump
    of eq. adv2d / adv3d with a = (1, ..., 1), degrees 3 and 5, on the one-task mesh of the
    study (2D: 60^2, table table:strong2d; 3D: 48^3, table table:advection3D), run to t = 1 on
    the FP64 path (the paper states no final time; a = (1, ..., 1) carries the bump once
    around the periodic domain, back to its start), with the L2 error (eq. l2relerror), the
    run time, the quality -log10(error x runtime) (eq. Quality) and the prediction's FP64
    rate over the upwind cells; beside them the paper's printed CPU figures.  The paper's nu
    is taken as dt = nu h / sum_d |a_d| (2D: 0.35, 3D: 0.2 per direction): read per direction
    instead (dt = nu h / max_d |a_d|) the 3D step's Fourier symbol has spectral radius 1.048
    at degree 3 and 2.9 at degree 5, and the runs blow up."""
    import torch
    ref = json.load(open(os.path.join(ROOT, "tests", "golden", f"paper_{dim}d_table.json")))
    rows = {}
    for M in (3, 5):
        n = (ref["mesh"],) * dim
        w = dict(flux="advection", dim=dim, n=n, M=M, vel=(1.0,) * dim, lo=(0.0,) * dim,
                 hi=(1.0,) * dim, cfl=ref["nu"] / dim)       # nu / sum_d |a_d|
        q0 = I.project_bump(w, M + 1, nq=16)
        X = I.project_bump(w, M + 2, nq=16)       # the exact solution at t = 1, degree M + 1
        s = R.Solver(dim, n, M, vel=w["vel"], cfl=w["cfl"])
        s.set_state(q0)
        nt = s.set_final_time(T_FINAL)
        p = s.profile_step(1)                     # one step, split per kernel (and warm-up)
        s.set_state(q0)
        s.set_final_time(T_FINAL)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        s.step(nt)                                # the run (its graph is captured first:
        b.record(s.stream)                        # host time, small against the steps)
        torch.cuda.synchronize()
        t_run = a.elapsed_time(b) * 1e-3
        e = s.l2_error(X)
        s.close()
        thS, cells = (M + 1) ** dim, int(np.prod(n))
        flops = 2.0 * thS * upwind_cells(w) * thS * cells   # the step's prediction: P-bar
        r = ref["rows"][str(M)]
        rows[str(M)] = {
            "steps": nt, "l2_error": e, "gpu_run_s": t_run, "quality": -np.log10(e * t_run),
            "ms_per_step": t_run / nt * 1e3, "predict_ms": p["predict_ms"],
            "correct_ms": p["correct_ms"],
            "predict_fp64_tflops": flops / (p["predict_ms"] * 1e-3) / 1e12,
            "paper_runtime_s": r["runtime_s"], "paper_cores": r["cores"],
            "paper_quality": r["quality"]}
        if "l2_error" in r:
            rows[str(M)]["paper_l2_error"] = r["l2_error"]
    return {"workload": f"adv{dim}d bump (eq. adv{dim}d), {ref['mesh']}^{dim}, "
                        f"a = (1, ..., 1), t = 1",
            "nu_paper": ref["nu"], "nu_per_direction": ref["nu"] / dim,
            "precision": "fp64", "rows": rows}


# ---------------------------------------------------------------------------------------
# the Newton path (nonlinear flux)
# ---------------------------------------------------------------------------------------
NL_WORKLOAD = "euler2d_n512_q2"
AUTOTUNE = [1]  # set from --autotune
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # FP32 FMA pipes x 2 flop x max SM clock
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12     # FP64 FMA: 2 per clock per SM


def newton_section(R, I, steps, cpu_cells):
    """The Newton prediction + correction of the 2D Euler vortex (512 x 512, Q2, m = 4): at full
    size the TF32 tensor-core block updates and the FP32 solves (both with the FP64 residual),
    FP64 solves on a 128 x 128 mesh of the same problem, and the oracle on a sample of cells
    (extrapolated per step)."""
    from oracle import nonlinear as ONL
    out = {"workload": NL_WORKLOAD}
    for tag, mesh, prec, peak in (("mixed_tf32", None, R.RIDG_PREC_MIXED_TF32, FP32_PEAK_TFLOPS),
                                  ("mixed_fp32", None, R.RIDG_PREC_MIXED_FP32, FP32_PEAK_TFLOPS),
                                  ("fp64_128x128", (128, 128), R.RIDG_PREC_FP64, FP64_PEAK_TFLOPS)):
        w = I.workload(NL_WORKLOAD, **({"n": mesh} if mesh else {}))
        s = R.Solver(2, w["n"], w["M"], flux="euler", cfl=w["cfl"], lo=w["lo"], hi=w["hi"],
                     gamma=w["gamma"], precision=prec)
        q = I.initial_state(w)
        s.set_state(q)
        if AUTOTUNE[0]:
            s.autotune()                         # the Newton grid for this precision
        s.profile_step(1)                        # warm-up
        p = s.profile_step(steps)
        info = s.info()
        grid = s.tuning()["newton_grid"]
        s.close()
        cells = int(np.prod(w["n"]))
        bs = 4 * (w["M"] + 1) ** 3               # unknowns of one region cell (m theta_T)
        iters = info["newton_iters_total"] / steps
        # algorithmic work of the block elimination (3 x 3 region, corners - edges - centre):
        # 9 block LUs (2/3 b^3), 17 block solves and 39 block updates (2 b^3 each) = 118 b^3
        flops = 118.0 * bs ** 3 * iters
        ach = flops / (p["predict_ms"] * 1e-3) / 1e12
        r = {"mesh": list(w["n"]), "ms_per_step": p["step_ms"], "predict_ms": p["predict_ms"],
             "correct_ms": p["correct_ms"],
             "value": cells * 4 * (w["M"] + 1) ** 2 / (p["step_ms"] * 1e-3),
             "unit": "element-DOF updates/s", "newton_iters_per_cell": iters / cells,
             "newton_iters_max": info["newton_iters_max"], "newton_grid_ctas": grid,
             "roofline": {"bound": "alu", "kernel": "newton_kernel", "achieved": ach, "peak": peak,
                          "unit": "TFLOP/s", "frac": ach / peak,
                          "traffic": (_recorded_traffic("newton_" + tag[6:], info["newton_iters_total"] / steps)
                                      if tag.startswith("mixed") else None),
                          "peak_source": "nominal: FMA pipes x 2 flop x 2.07 GHz"}}
        if tag == "mixed_tf32":
            # the 56 block products alone (2 b^3 flop each: 112 of the 118 b^3) on the TF32
            # tensor cores: TF32 peak = the measured BF16 peak x the nominal TF32 / BF16 ratio
            tf32_peak = _peaks()[1] * 0.5
            upd = 112.0 * bs ** 3 * iters / (p["predict_ms"] * 1e-3) / 1e12
            r["tensor"] = {"kernel": "newton_kernel (block updates)", "achieved": upd,
                           "peak": tf32_peak, "unit": "TFLOP/s", "frac": upd / tf32_peak,
                           "peak_source": "measured BF16 x nominal TF32/BF16 (1/2)"}
        out[tag] = r
    out["accuracy"] = newton_accuracy(R, I)
    # the oracle: Newton prediction of a sample of cells and the correction of the whole
    # mesh is not needed for a per-cell rate; extrapolated to every cell of the step
    w = I.workload(NL_WORKLOAD, n=(32, 32))
    q = I.initial_state(w)
    from oracle import linear as OL
    dt, _ = OL.time_step(w, ONL.max_speed(q, w))
    cells = np.arange(cpu_cells)
    t0 = time.perf_counter()
    ONL.newton_predict(q, w, dt, cells=cells)
    per_cell = (time.perf_counter() - t0) / cpu_cells
    full = 512 * 512
    out["cpu_oracle"] = {"kind": "oracle", "cores": os.cpu_count(),
                         "seconds_per_cell": per_cell,
                         "value": full * 4 * 9 / (per_cell * full),
                         "unit": "element-DOF updates/s",
                         "sample": f"Newton predictions of {cpu_cells} cells of the vortex "
                                   "(numpy, all host cores), extrapolated to 512 x 512"}
    return out


def newton3d_section(R, I, cpu=True):
    """The 3D nonlinear prediction (3D Burgers, degree 1, smooth seeded data): one step at 32^3
    with FP32 region solves (FP64 residual and update) and at 12^3 in FP64, each with the
    rate of its dense per-region LU (2/3 n^3 flop per factorisation, n = 27 theta_T = 432)
    against the FP32 / FP64 pipe, and the oracle's per-region time on the host."""
    import torch
    from oracle import linear as OL
    from oracle import nonlinear as ONL

    def data(n):
        w = dict(flux="burgers", dim=3, n=(n,) * 3, M=1, lo=(0.0,) * 3, hi=(1.0,) * 3, cfl=0.3)
        f = lambda x, y, z: (0.3 + 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
                             * np.sin(2 * np.pi * z) + 0.05 * np.cos(2 * np.pi * (x + z)))
        return w, np.ascontiguousarray(I.project_tensor(f, w, 2)[:, 0, :])

    out = {"workload": "burgers3d Q1, smooth data (sines)", "solver": "dense per-region LU"}
    for tag, n, prec, peak in (("mixed_fp32", 32, R.RIDG_PREC_MIXED_FP32, FP32_PEAK_TFLOPS),
                               ("fp64", 12, R.RIDG_PREC_FP64, FP64_PEAK_TFLOPS)):
        w, q = data(n)
        s = R.Solver(3, w["n"], 1, flux="burgers", cfl=w["cfl"], precision=prec,
                     newton_max_iters=8)
        s.set_state(q)
        s.profile_step(1)                         # warm-up
        s.set_state(q)
        p = s.profile_step(1)
        info = s.info()
        s.close()
        cells = n ** 3
        flops = 2.0 / 3.0 * 432.0 ** 3 * info["newton_iters_total"]
        ach = flops / (p["predict_ms"] * 1e-3) / 1e12
        out[tag] = {"mesh": [n] * 3, "ms_per_step": p["step_ms"], "predict_ms": p["predict_ms"],
                    "correct_ms": p["correct_ms"], "value": cells * 8 / (p["step_ms"] * 1e-3),
                    "unit": "element-DOF updates/s",
                    "newton_iters_per_cell": info["newton_iters_total"] / cells,
                    "roofline": {"bound": "alu", "kernel": "newton3_kernel (LU flops)",
                                 "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                 "frac": ach / peak, "traffic": None,
                                 "peak_source": "nominal: FMA pipes x 2 flop x 2.07 GHz"}}
    if cpu:
        w, q = data(12)
        dt, _ = OL.time_step(w, ONL.max_speed(q, w))
        t0 = time.perf_counter()
        ONL.newton_predict(q, w, dt, cells=np.arange(8), max_iters=8)
        per = (time.perf_counter() - t0) / 8
        out["cpu_oracle"] = {"kind": "oracle", "cores": os.cpu_count(), "seconds_per_cell": per,
                             "value": 8 / per, "unit": "element-DOF updates/s",
                             "sample": "Newton predictions of 8 cells (numpy, host cores)"}
    return out


def newton_accuracy(R, I):
    """The config's equal-accuracy check on a mesh the oracle can run to t = 1: the Euler
    vortex at Q2 on 32^2 (27 steps) with each Newton precision, L2 error against the
    translated vortex (eq. l2relerror) beside the oracle's (tests/golden)."""
    from oracle import error as OE
    g = _golden().get("euler2d_n32_q2")
    if g is None:
        return None
    w = I.workload(NL_WORKLOAD, n=(32, 32))
    X = I.exact_coefficients(w, 1.0)
    out = {"workload": "euler2d Q2 on 32^2, t = 1", "steps": g["steps"],
           "l2_error_oracle": g["l2_error"]}
    for tag, prec in (("mixed_tf32", R.RIDG_PREC_MIXED_TF32), ("mixed_fp32", R.RIDG_PREC_MIXED_FP32),
                      ("fp64", R.RIDG_PREC_FP64)):
        s = R.Solver(2, w["n"], w["M"], flux="euler", cfl=w["cfl"], lo=w["lo"], hi=w["hi"],
                     gamma=w["gamma"], precision=prec)
        s.set_state(I.initial_state(w))
        s.set_dt(g["dt"])
        s.step(g["steps"])
        s.sync()
        e = OE.l2_relative_error(s.get_state(), X, w["M"], 2, m=4)
        s.close()
        out[tag] = {"l2_error": e, "equal_accuracy": bool(e <= 1.05 * g["l2_error"])}
    return out


def ensemble_accuracy(R, I, prec):
    """The ensemble's equal-accuracy check on instances capped at 16^2 (the oracle's errors are
    on record for them, tests/golden): one batched run, each instance to half its shock time
    in a common step count; the worst ratio of an instance's L2 error against the exact
    pre-shock solution to the oracle's."""
    from oracle import error as OE
    g = _golden().get("burgers_ens16")
    if g is None:
        return None
    ens = [dict(w, n=(min(w["n"][0], 16), min(w["n"][1], 16))) for w in I.burgers_ensemble()]
    b = R.ridg_batch_create([R.make_mesh(2, w["n"]) for w in ens], [w["M"] for w in ens],
                            R.make_flux("burgers"), ens[0]["cfl"], R.make_options(precision=prec))
    N = g["steps"]
    for i, (w, T) in enumerate(zip(ens, g["T"])):
        h = R.ridg_batch_instance(b, i)
        R.ridg_set_state(h, I.initial_state(w))
        R.ridg_set_dt(h, T / N)
    R.ridg_batch_step(b, N)
    R.ridg_batch_sync(b)
    errs = []
    for i in g["instances"]:            # the instances the oracle's errors are on record for
        w, T = ens[i], g["T"][i]
        q = np.empty((int(np.prod(w["n"])), (w["M"] + 1) ** 2))
        R.ridg_get_state(R.ridg_batch_instance(b, i), q)
        errs.append(OE.l2_relative_error(q, I.exact_coefficients(w, T), w["M"], 2))
    R.ridg_batch_destroy(b)
    ratios = [e / o for e, o in zip(errs, g["l2_error"])]
    return {"workload": "burgers ensemble capped at 16^2, T_i = t_shock_i / 2 (all 64 "
                        "instances in the batch; the first four of each degree checked "
                        "against the oracle)", "steps": N,
            "l2_error_max": max(errs), "l2_error_oracle_max": max(g["l2_error"]),
            "worst_ratio_to_oracle": max(ratios), "equal_accuracy": bool(max(ratios) <= 1.05)}


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        rows = []
        try:
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def _recorded_traffic(prec_name, units=None):
    """DRAM bytes per launch of the dominant kernel, from the committed ncu summaries under
    profiles/ (a line `roofline-traffic: <name> <source> sha256_16=<h> dram_bytes=<n>
    [units=<u>]`), used only while that kernel source is unchanged since the capture (else
    None).  A capture of a smaller case carries the units (e.g. region-iterations) it
    processed; its bytes are scaled to `units` of this launch."""
    import glob
    import hashlib
    for p in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(p):
            f = line.split()
            if len(f) < 5 or f[0] != "roofline-traffic:" or f[1] != prec_name:
                continue
            kv = dict(x.split("=", 1) for x in f[3:])
            src = os.path.join(ROOT, "paper_2101_01231_gb300", "csrc", f[2])
            if not os.path.exists(src):
                return None
            h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
            if h != kv.get("sha256_16"):
                return None
            b = int(kv["dram_bytes"])
            if "units" in kv:
                return None if units is None else b / int(kv["units"]) * units
            return b
    return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


def linear_arm(R, I, w, args, ws, flush, clocks=None, steps=None):
    """One linear-advection workload: the digit-count gate, the timed mixed path (whole steps
    through ridg_step and the per-kernel split), the FP64 path beside it, the end-to-end
    number through the C ABI with host buffers, the accuracy figures and the roofline of the
    dominant kernel."""
    import torch
    import torch.distributed as dist
    steps = steps or args.steps
    noisy = w.get("ic") == "sin+noise"
    prec = {"fp64": R.RIDG_PREC_FP64, "mixed": R.RIDG_PREC_MIXED_BF16}
    prec_name = args.precision if args.precision != "auto" else "mixed"
    chosen = [args.slices]

    def make(pname, slices=None):
        return R.Solver(w["dim"], w["n"], w["M"], vel=w["vel"], cfl=w["cfl"], lo=w["lo"],
                        hi=w["hi"], precision=prec[pname],
                        slices=chosen[0] if slices is None else slices)

    if prec_name == "mixed":
        try:
            make("mixed").close()
        except R.RidgError:
            prec_name = "fp64"
    cells = int(np.prod(w["n"]))
    thS = (w["M"] + 1) ** w["dim"]
    K = upwind_cells(w) * thS
    dof = cells * thS
    q0 = I.initial_state(w)
    exact = None if noisy else I.exact_coefficients(w, T_FINAL)

    def accuracy(pname, slices=None):
        """L2 error against the exact solution at t = 1: for the noisy data integrated exactly
        on the sub-box overlaps of the carried piecewise polynomial, else eq. l2relerror
        against the exact solution's Q(M+1) projection (ridg_l2_error)."""
        s = make(pname, slices)
        s.set_state(q0)
        nt = s.set_final_time(T_FINAL)
        s.step(nt)
        s.sync()
        e = (I.shifted_polynomial_error(w, q0, s.get_state(), T_FINAL) if noisy
             else s.l2_error(exact))
        s.close()
        return e, nt

    def timed(pname, nsteps, warmup, ck=None):
        """Whole steps through ridg_step (the captured graph: prediction and correction back to
        back), timed with CUDA events on the handle's stream, L2 flushed before each; then
        the per-kernel split (prediction / correction, events around each launch) under the
        same flush."""
        s = make(pname)
        s.set_state(q0)
        s.set_final_time(T_FINAL)
        for _ in range(warmup):
            with torch.cuda.stream(s.stream):
                flush.fill_(1.0)
            s.step(1)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        if ck:
            ck.start()
        # a GPU-side wait (outside every timed interval) lets the host queue the flushes,
        # events and steps ahead of the GPU, so no host launch latency falls between an
        # event pair (on a slow host it otherwise does: +27 us per step seen once)
        with torch.cuda.stream(s.stream):
            torch.cuda._sleep(int(2.0e9 * min(0.2, 1e-4 * nsteps + 0.02)))
        evs = []
        for i in range(nsteps):
            with torch.cuda.stream(s.stream):
                flush.fill_(float(i))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s.stream)
            s.step(1)
            b.record(s.stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ckr = ck.stop() if ck else None
        tt = sum(a.elapsed_time(b) for a, b in evs) / nsteps
        nsplit = min(nsteps, 50)
        tp = tc = 0.0
        for i in range(nsplit):
            with torch.cuda.stream(s.stream):
                flush.fill_(float(i))
            p = s.profile_step(1)
            tp += p["predict_ms"]
            tc += p["correct_ms"]
        torch.cuda.synchronize()
        return s, tt, tp / nsplit, tc / nsplit, ckr

    # the mixed form's digit count: the fewest slices whose L2 error against the exact
    # solution at t = 1 is within 1.05x of the FP64 path's (which matches the oracle's)
    sweep = None
    e64, nt = accuracy("fp64")
    if prec_name == "mixed" and args.slices == 0:
        sweep = {}
        for S in range(3, 8):
            try:
                sweep[S] = accuracy("mixed", S)[0]
            except R.RidgError:
                break
            if sweep[S] <= 1.05 * e64:
                chosen[0] = S
                break
    tuning = None
    if args.autotune and prec_name == "mixed":
        # the autotuner times the launch choices on this workload's state; the timed
        # handles below read its choices from the library's cache
        st = make("mixed")
        st.set_state(q0)
        st.autotune()
        tuning = st.tuning()
        st.close()
    hbm, bf16, src = _peaks()
    s, ms_step, ms_pred, ms_corr, ck = timed(prec_name, steps, args.warmup, clocks)
    slices_used = s.info()["slices"]
    ms_step = max_over_ranks(ms_step, ws, "cuda")

    # end to end through the C ABI with host buffers: H2D state, one step, D2H state
    qh = torch.from_numpy(q0.copy()).pin_memory().numpy()
    n_e2e = min(steps, 20)
    for _ in range(3):
        s.set_state(qh)
        s.step(1)
        s.get_state(qh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        s.set_state(qh)
        s.step(1)
        s.get_state(qh)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / n_e2e, ws, "cuda")
    s.close()

    predict_full = None
    if prec_name == "mixed" and w["dim"] == 3:
        predict_full = time_predict(R, I, w, make, q0, slices_used, hbm, bf16)
    fp64 = None
    if prec_name != "fp64":
        s2, ms64, mp64, mc64, _ = timed("fp64", max(10, steps // 5), args.warmup)
        s2.close()
        fp64 = {"ms_per_step": ms64, "value": dof / (ms64 * 1e-3), "predict_ms": mp64,
                "correct_ms": mc64}
    err = accuracy(prec_name)[0] if prec_name != "fp64" else e64

    # Algorithmic work per launch.  Prediction (time mean): 2 theta_S K flop per cell (K =
    # theta_S x the upwind region cells; the other region cells' operator columns are exactly
    # zero) and its bytes: read Q (8 theta_S B per cell), write its outputs -- W-bar (8
    # theta_S), or in the mixed path the fused step operator's outputs as double-float pairs:
    # the volume term and the upwind face traces, theta_S + 2 (M + 1) in 2D and theta_S +
    # 3 (M + 1)^2 in 3D where the digits fit the GEMM (3D: slices x padded rows <= 256), else
    # W-bar.  Correction: read those outputs, read and write Q (16 theta_S).
    flops_pred = 2.0 * thS * K * cells
    nb_ = w["M"] + 1
    if prec_name == "fp64":
        nfused = thS
    elif w["dim"] == 2:
        nfused = thS + 2 * nb_
    else:
        nf3 = thS + 3 * nb_ * nb_
        nfused = nf3 if slices_used * (32 if nf3 <= 32 else 64) <= 256 else thS
    npad = 32 if nfused <= 32 else 64
    bytes_pred = (8.0 * thS + 8.0 * nfused) * cells
    bytes_corr = (8.0 * nfused + 16.0 * thS) * cells
    if prec_name == "fp64":
        # FP64 FMA pipe: 152 SMs x 2 FP64 FMA / clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)
        roof = {"bound": "alu", "kernel": "predict_fp64",
                "achieved": flops_pred / (ms_pred * 1e-3) / 1e12, "peak": 1.25, "unit": "TFLOP/s",
                "traffic": _recorded_traffic("fp64"),
                "peak_source": "nominal FP64 rate (152 SMs x 4 flop/clk x 2.07 GHz)"}
    else:
        S_ = slices_used
        # executed on the tensor pipe: digit pairs x padded outputs x padded K (each region
        # cell's modes padded to a multiple of 16)
        kpad = upwind_cells(w) * ((thS + 15) // 16) * 16
        executed = 2.0 * (S_ * (S_ + 1) // 2) * npad * kpad * cells
        tag = "mixed3" if w["dim"] == 3 else "mixed"
        gemm = {"bound": "hbm", "kernel": f"{tag}_gemm (prediction)", "ms": ms_pred,
                "achieved": bytes_pred / (ms_pred * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "traffic": _recorded_traffic(tag + "gemm", cells),
                "peak_source": f"HBM copy, {src}",
                "algorithmic_bytes_per_cell": bytes_pred / cells, "outputs_per_cell": nfused,
                "tensor_executed_tflops": executed / (ms_pred * 1e-3) / 1e12,
                "tensor_peak_tflops": bf16,
                "algorithmic_tflops": flops_pred / (ms_pred * 1e-3) / 1e12}
        # (3D: mixed3_fcorrect reads the fused step operator's outputs, mixed3_correct the
        # time means where those digits do not fit the GEMM)
        ctag = tag + ("_fcorrect" if w["dim"] == 3 and nfused > thS else "_correct")
        corr = {"bound": "hbm", "kernel": f"{ctag} (correction)", "ms": ms_corr,
                "achieved": bytes_corr / (ms_corr * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "traffic": _recorded_traffic(ctag.replace("_correct", "corr").replace("_", ""), cells),
                "peak_source": f"HBM copy, {src}",
                "algorithmic_bytes_per_cell": bytes_corr / cells}
        for r in (gemm, corr):
            r["frac"] = r["achieved"] / r["peak"]
        roof = dict(corr if ms_corr >= ms_pred else gemm)
        roof["other_kernel"] = gemm if ms_corr >= ms_pred else corr
        # the whole step against the bytes it fundamentally moves (Q in and out)
        roof["step_bytes_per_cell"] = 16.0 * thS
        roof["step_frac"] = 16.0 * thS * cells / (ms_step * 1e-3) / 1e9 / hbm
    roof["frac"] = roof["achieved"] / roof["peak"]
    gate_ref = e64
    out = {
        "workload": w["name"], "cells": cells, "order": w["M"], "theta_s": thS,
        "precision": prec_name, "slices": slices_used if prec_name == "mixed" else None,
        "steps": steps, "ms_per_step": ms_step, "value": ws * dof / (ms_step * 1e-3),
        "unit": "element-DOF updates/s", "steps_to_T": nt,
        "kernels_ms": {"predict": ms_pred, "correct": ms_corr}, "autotune": tuning,
        "fp64_path": fp64, "roofline": roof, "predict_full": predict_full,
        "e2e": {"value": ws * dof / e2e_s, "unit": "element-DOF updates/s",
                "h2d_bytes_per_step": int(q0.nbytes), "d2h_bytes_per_step": int(q0.nbytes)},
        "accuracy": {"T": T_FINAL,
                     "measure": ("exact: the noisy piecewise polynomial carried by a t, "
                                 "integrated on the sub-box overlaps") if noisy
                                else "eq. l2relerror against the exact solution's Q(M+1) projection",
                     "l2_error": err, "l2_error_fp64_gpu": e64,
                     "equal_accuracy": bool(err <= 1.05 * gate_ref),
                     "slices_sweep_l2_error": ({str(k): v for k, v in sweep.items()}
                                               if sweep else None)},
        "clocks": ck,
    }
    gold = _golden()
    if w["name"] in gold and not noisy:
        g = gold[w["name"]]
        out["accuracy"]["l2_error_oracle"] = g["l2_error"]
        out["accuracy"]["equal_accuracy_vs_oracle"] = bool(err <= 1.05 * g["l2_error"])
    elif noisy and "adv3d_n24_q2_noise" in gold:
        # the oracle at full size would take hours (~44 s per step on the host): its error is
        # on record for the same data on a 24^3 mesh, where the GPU paths are checked against
        # it by the GPU tests; at full size the FP64 GPU path (per-step parity 1e-12) stands in
        out["accuracy"]["l2_error_oracle_24cubed"] = gold["adv3d_n24_q2_noise"]["l2_error"]
    return out


def time_predict(R, I, w, make, q0, slices, hbm, bf16, reps=10):
    """ridg_predict of every cell's full space-time prediction (all theta_T rows of the
    operator: the full space-time contraction of 3D advection, Q2) through the C ABI into a
    device buffer, timed with CUDA events on the handle's stream: its executed tensor rate
    (digit-pair products, outputs and K padded) against the BF16 peak, its algorithmic rate
    (2 theta_T K flop per cell) and the bytes it must move (Q in, W out in FP64)."""
    import torch
    s = make("mixed", slices)
    s.set_state(q0)
    cells = int(np.prod(w["n"]))
    thS = (w["M"] + 1) ** w["dim"]
    thT = thS * (w["M"] + 1)
    K = upwind_cells(w) * thS
    Wd = torch.empty(cells, thT, dtype=torch.float64, device="cuda")
    s.predict(Wd)                                 # warm-up (digit planes, attributes)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s.stream)
    for _ in range(reps):
        s.predict(Wd)
    b.record(s.stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    s.close()
    # executed: P's theta_T rows in blocks of 64 (32 when slices x 64 > 256), one GEMM launch
    # each: S (S + 1) / 2 digit pairs x the block's padded rows (32 or 64) x the upwind cells'
    # padded modes, per cell
    R = 64 if slices * 64 <= 256 else 32
    blocks = [min(R, thT - r0) for r0 in range(0, thT, R)]
    npads = sum(32 if b <= 32 else 64 for b in blocks)
    kpad = upwind_cells(w) * ((thS + 15) // 16) * 16
    executed = 2.0 * (slices * (slices + 1) // 2) * npads * kpad * cells
    return {"kernel": f"mixed3_gemm x {len(blocks)} row blocks and their FP64 rows (ridg_predict)",
            "ms": ms,
            "tensor_executed_tflops": executed / (ms * 1e-3) / 1e12, "tensor_peak_tflops": bf16,
            "tensor_frac": executed / (ms * 1e-3) / 1e12 / bf16,
            "algorithmic_tflops": 2.0 * thT * K * cells / (ms * 1e-3) / 1e12,
            "hbm_gbs": 8.0 * (thS + thT) * cells / (ms * 1e-3) / 1e9, "hbm_peak_gbs": hbm}


def run_ours(args):
    import torch
    import torch.distributed as dist

    AUTOTUNE[0] = args.autotune
    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2101_01231_gb300 import inputs as I
    from paper_2101_01231_gb300 import ridg as R

    w = I.workload(args.workload)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        gpu_id = str(torch.cuda.current_device())
    head = linear_arm(R, I, w, args, ws, flush, Clocks(gpu_id))
    acc = head["accuracy"]
    line = {
        "metric": "element-DOF updates/s per RIDG step",
        "value": head["value"], "unit": "element-DOF updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head["precision"] == "fp64" else "bf16x{}+f64".format(head["slices"]),
        "data": "synthetic",
        "config": {"workload": w["name"], "cells": head["cells"], "order": w["M"],
                   "theta_s": head["theta_s"], "precision": head["precision"],
                   "steps_to_T": head["steps_to_T"],
                   "l2_flush": "state (191 MB) larger than L2, and a 256 MB rewrite before each "
                               "timed step" if w["dim"] == 3 else
                               "256 MB rewrite before each timed step",
                   "l2_error": acc["l2_error"], "l2_error_fp64_gpu": acc["l2_error_fp64_gpu"],
                   "l2_error_oracle": acc.get("l2_error_oracle",
                                              acc.get("l2_error_oracle_24cubed")),
                   "equal_accuracy": acc["equal_accuracy"],
                   "slices_sweep_l2_error": acc["slices_sweep_l2_error"],
                   "error_measure": acc["measure"]},
        "kernels_ms": head["kernels_ms"],
        "autotune": head["autotune"],
        "predict_full": head["predict_full"],
        "fp64_path": head["fp64_path"],
        "roofline": head["roofline"],
        "e2e": head["e2e"],
        "gpu_launches": 2 * args.steps,
        "clocks": head["clocks"],
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = (cpu_oracle_sampled(w, I.initial_state(w)) if w["dim"] == 3
                                else cpu_oracle(w, args.cpu_seconds))
    if args.adv2d_steps > 0 and args.workload != WORKLOAD_2D:
        w2 = I.workload(WORKLOAD_2D)
        line["adv2d"] = linear_arm(R, I, w2, args, ws, flush, None, steps=args.adv2d_steps)
        if rank == 0 and not args.no_cpu_baseline and ws == 1:
            line["adv2d"]["cpu_oracle"] = cpu_oracle(w2, args.cpu_seconds)
    if args.newton_steps > 0:
        line["newton"] = newton_section(R, I, args.newton_steps, 8 if args.no_cpu_baseline else 16)
        line["newton3d"] = newton3d_section(R, I, cpu=not args.no_cpu_baseline)
    if args.adv1d_reps > 0:
        line["adv1d"] = adv1d_section(R, I, args.adv1d_reps)
    if args.paper1d > 0:
        line["paper1d"] = paper1d_section(R, I)
    if args.paper2d > 0:
        line["paper2d"] = paper_bump_section(R, I, 2)
    if args.paper3d > 0:
        line["paper3d"] = paper_bump_section(R, I, 3)
    if args.ensemble_steps > 0 and ws <= 64:
        line["ensemble"] = ensemble_section(R, I, args.ensemble_steps, 4, rank, ws)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
