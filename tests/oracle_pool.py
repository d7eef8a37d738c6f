"""Runs of the nonlinear oracle over several host processes (test helper).

The oracle's Newton prediction is independent per cell, so a step's cells are split
over a spawn-started pool (each worker single-threaded), then the correction runs on the
whole mesh.  Arithmetic is the oracle's, unchanged."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_THREADS = dict(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def _predict(args):
    from oracle import nonlinear as NL
    Q, w, dt, cells, alpha, max_iters, tol = args
    return NL.newton_predict(Q, w, dt, cells=cells, alpha=alpha, max_iters=max_iters, tol=tol,
                             return_iters=True)


class Pool:
    def __init__(self, procs: int | None = None):
        self.procs = procs or min(8, os.cpu_count() or 1)
        old = {k: os.environ.get(k) for k in _THREADS}
        os.environ.update(_THREADS)   # inherited by the spawned workers
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs)
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.pool.terminate()
        self.pool.join()

    def predict(self, Q, w, dt, alpha="frozen", max_iters=4, tol=1e-10):
        chunks = np.array_split(np.arange(Q.shape[0]), 2 * self.procs)
        res = self.pool.map(_predict, [(Q, w, dt, c, alpha, max_iters, tol) for c in chunks])
        W = np.concatenate([r[0] for r in res])
        iters = np.concatenate([r[1] for r in res])
        conv = np.concatenate([r[2] for r in res])
        return W, iters, conv

    def run(self, Q0, w, dt, nsteps, alpha="frozen", max_iters=4, tol=1e-10):
        """nsteps oracle RIDG steps; returns (Q, unconverged region-steps)."""
        from oracle import nonlinear as NL
        Q, unconv = Q0.copy(), 0
        for _ in range(nsteps):
            W, _, conv = self.predict(Q, w, dt, alpha, max_iters, tol)
            unconv += int((~conv).sum())
            Q = NL.correct(Q, W, w, dt, pointwise=alpha == "point")
        return Q, unconv
